"""The library's schedule of the temporal decomposition (Sec. 3.3, Eq. 10;
nlinv_stream_source / nlinv_stream_schedule, host-only C functions) matches
the oracle's schedule and never reads a frame finished in the same launch
(CPU only: the library loads without a GPU and these calls launch nothing)."""
import pytest

import oracle as O
from paper_1701_08361_gb300 import nlinv as L
from paper_1701_08361_gb300 import stream as ST


def test_sources_match_oracle():
    for D in (1, 2, 3, 11):
        for l in (0, 2, 5):
            for n in range(40):
                assert L.nlinv_stream_source(n, D, l) == O.source_frame(n, D, l)
                assert ST.source(n, D, l) == O.source_frame(n, D, l)


def test_groups_cover_frames_once_and_respect_dependencies():
    for D in (1, 3, 10, 11):
        for l in (0, 5):
            for nf in (1, 7, 32, 60):
                gs = ST.groups(nf, D, l)
                flat = [n for g in gs for n in g]
                assert flat == list(range(nf))
                done = set()
                for g in gs:
                    assert len(g) <= max(D, 1)
                    for n in g:
                        s = ST.source(n, D, l)
                        assert s < 0 or s in done
                    done.update(g)


@pytest.mark.parametrize("NF,D,WU", [(14, 3, 2), (40, 11, 5), (9, 1, 0), (8, 4, 0)])
def test_last_step_regulariser_is_the_previous_frame(NF, D, WU):
    """With last_from_prev, every frame whose source is not n - 1 is given
    x^_{n-1} for its last Newton step, and that frame is either finished in an
    earlier launch group or an EARLIER frame of the same group (the only
    in-call reference nlinv_batch accepts); sources are always in earlier
    groups.  Without the option no frame gets one."""
    grp, src, last = L.nlinv_stream_schedule(NF, D, WU, True)
    for n in range(NF):
        assert src[n] == O.source_frame(n, D, WU)
        assert src[n] < 0 or grp[src[n]] < grp[n]
        if n == 0 or src[n] == n - 1:
            assert last[n] == -1
        else:
            assert last[n] == n - 1
            assert grp[n - 1] < grp[n] or (grp[n - 1] == grp[n] and n - 1 < n)
    _, _, last0 = L.nlinv_stream_schedule(NF, D, WU, False)
    assert all(v == -1 for v in last0)


def test_schedule_rejects_bad_arguments():
    for args in ((5, 0, 0), (5, 1, -1), (-1, 1, 0)):
        with pytest.raises(L.NlinvError):
            L.nlinv_stream_schedule(*args)
    for args in ((-1, 1, 0), (3, 0, 0), (3, 1, -2)):
        with pytest.raises(L.NlinvError):
            L.nlinv_stream_source(*args)
