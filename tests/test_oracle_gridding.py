"""Pins of the oracle's convolution gridding (the preprocessing stage of
Sec. 3.1 in its Kaiser-Bessel form, oracle.grid_data_kb) against what the
mathematics fixes (CPU only):

* the closed-form transform of the kernel (kb_ft) against numerical
  quadrature of the kernel itself;
* the gridded data against the exact adjoint NDFT (oracle.grid_data, itself
  pinned against the loop-built NDFT matrix) within the kernel-width error
  bound, on twofold and non-twofold grids;
* the error falling geometrically with the kernel width W (a dropped
  deapodisation, a wrong centre or a wrong sign fails this by orders of
  magnitude).
"""
import numpy as np
import pytest
from scipy import integrate

import oracle as O
import synth as S


@pytest.mark.parametrize("W", [4, 6, 8])
def test_kb_transform_closed_form_matches_quadrature(W):
    beta = O.kb_beta(W, 2.0)
    for t in (0.0, 0.05, 0.17, 0.25, 0.33):
        num, _ = integrate.quad(lambda u: O.kb_kernel(u, W, beta) * np.cos(2 * np.pi * u * t),
                                -W / 2, W / 2, epsabs=0, epsrel=1e-13, limit=200)
        assert abs(O.kb_ft(t, W, beta) - num) <= 1e-10 * abs(num)


def test_kb_kernel_support_and_peak():
    beta = O.kb_beta(6, 2.0)
    assert O.kb_kernel(0.0, 6, beta) == pytest.approx(np.i0(beta), rel=1e-15)
    assert O.kb_kernel(3.0, 6, beta) == pytest.approx(1.0)           # I0(0) at the edge
    assert O.kb_kernel(3.0001, 6, beta) == 0.0 and O.kb_kernel(-3.5, 6, beta) == 0.0


# (N, G, W, bound): the measured error of W = 6 / 8 is 2e-6..7e-6 / 1e-8..8e-8
@pytest.mark.parametrize("N,G,W,bound", [(16, 32, 6, 2e-5), (32, 64, 6, 2e-5), (20, 56, 6, 1e-5),
                                         (24, 72, 6, 1e-5), (16, 32, 8, 3e-7), (20, 56, 8, 1e-7)])
def test_kb_gridding_matches_exact_adjoint_ndft(N, G, W, bound):
    kx, ky = S.radial_trajectory(N, 9, 5, 1)
    y = S.random_complex((2, len(kx)), 3)
    exact = O.grid_data(kx, ky, y, N, G)
    got = O.grid_data_kb(kx, ky, y, N, G, W)
    assert np.linalg.norm(got - exact) <= bound * np.linalg.norm(exact)


def test_kb_gridding_error_falls_with_kernel_width():
    N, G = 16, 32
    rng = np.random.default_rng(9)
    kx, ky = rng.uniform(-0.5, 0.5, 300), rng.uniform(-0.5, 0.5, 300)
    y = S.random_complex((1, 300), 11)
    exact = O.grid_data(kx, ky, y, N, G)
    errs = [np.linalg.norm(O.grid_data_kb(kx, ky, y, N, G, W) - exact) / np.linalg.norm(exact)
            for W in (3, 4, 5, 6, 7, 8)]
    for a, b in zip(errs, errs[1:]):
        assert b < a / 4, errs
    assert errs[-1] < 1e-6
