"""Temporal decomposition of a stream of frames (Sec. 3.3, Eq. 10).

The schedule itself lives in the C library (nlinv_stream_source,
nlinv_run_streams): frames 0..l of a stream are reconstructed in order,
afterwards D frames are in flight together and each starts from (and is
regularised towards) the last frame of the previous group; with the paper's
exception (last_from_prev) the last Newton step of frame n is regularised
towards x^_{n-1}.  This module only re-exports the schedule for callers and
lists a stream's launch groups.
"""
from __future__ import annotations

from . import nlinv as L


def source(n: int, delay: int, warmup: int) -> int:
    """Index of the frame whose x^ frame n starts from (-1: rho = 1, c = 0)."""
    return L.nlinv_stream_source(n, delay, warmup)


def groups(nframes: int, delay: int, warmup: int):
    """Launch groups of one stream, as the library forms them: [[0], [1], ...,
    [warmup], then runs of `delay` frames]."""
    grp, _, _ = L.nlinv_stream_schedule(nframes, delay, warmup)
    out = [[] for _ in range(max(grp) + 1 if grp else 0)]
    for n, g in enumerate(grp):
        out[g].append(n)
    return out


def run(streams, stream=None):
    """Reconstruct several independent streams together (nlinv_run_streams).

    streams: list of dicts {plan, Y: list of device tensors, turns: list of
    ints, delay, warmup, x: device tensor [nframes, n_x] for the outputs,
    img: optional device tensor [nframes, N*N], last_from_prev: optional
    bool}.
    """
    L.nlinv_run_streams(streams, stream)
