"""Pins of the oracle's temporal median filter (post-processing stage of
Sec. 3.1) against a brute-force per-pixel sort and closed cases (CPU only)."""
import numpy as np
import pytest

import oracle as O
import synth as S


@pytest.mark.parametrize("T", [1, 3, 5, 7])
def test_median_is_the_middle_of_the_sorted_window(T):
    imgs = S.random_complex((T, 6, 5), 13 + T)
    got = O.temporal_median(imgs)
    for y in range(6):
        for x in range(5):
            vals = sorted(float(np.abs(imgs[t, y, x])) for t in range(T))
            assert got[y, x] == vals[T // 2]


def test_median_closed_cases():
    a = S.random_complex((4, 4), 3)
    # a window of one frame is the magnitude; a constant window is its value
    np.testing.assert_array_equal(O.temporal_median(a[None]), np.abs(a))
    np.testing.assert_array_equal(O.temporal_median(np.stack([a, a, a])), np.abs(a))
    # a monotone sequence of magnitudes gives the middle frame; an outlier frame is removed
    seq = np.stack([a * s for s in (1.0, 2.0, 3.0, 4.0, 5.0)])
    np.testing.assert_allclose(O.temporal_median(seq), 3.0 * np.abs(a), rtol=1e-15)
    spike = np.stack([a, a, 100.0 * a])
    np.testing.assert_array_equal(O.temporal_median(spike), np.abs(a))
    with pytest.raises(AssertionError):
        O.temporal_median(np.stack([a, a]))
