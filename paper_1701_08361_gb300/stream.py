"""Host-side schedule of the temporal decomposition (Sec. 3.3, Eq. 10) and a
driver that runs it through the C ABI.

Frames 0..l of a stream are reconstructed strictly in order; afterwards D
frames are in flight together and each starts from (and is regularised
towards) the most recent frame finished when its group starts -- the last
frame of the previous group.  With the paper's exception (last_from_prev),
the last Newton step of frame n is regularised towards x^_{n-1} instead, so
inside a group that step waits for the frame before it (the library resolves
the wait from the buffers).  This module only decides which frame goes into
which launch and which earlier outputs it reads; all computation happens in
nlinv_frame / nlinv_batch.
"""
from __future__ import annotations

import torch

from . import nlinv as L


def source(n: int, delay: int, warmup: int) -> int:
    """Index of the frame whose x^ frame n starts from (-1: rho = 1, c = 0)."""
    if n <= warmup:
        return n - 1
    return warmup + ((n - warmup - 1) // delay) * delay


def groups(nframes: int, delay: int, warmup: int):
    """Launch groups of one stream: [[0], [1], ..., [warmup], then runs of
    `delay` frames]; every frame's source is finished in an earlier group."""
    out = [[n] for n in range(min(nframes, warmup + 1))]
    n = warmup + 1
    while n < nframes:
        out.append(list(range(n, min(n + delay, nframes))))
        n += delay
    return out


def run(streams, stream=None):
    """Reconstruct several independent streams together.

    streams: list of dicts {plan, Y: list of device tensors, turns: list of
    ints, delay, warmup, x: device tensor [nframes, n_x] for the outputs,
    img: optional device tensor [nframes, N*N], last_from_prev: optional
    bool}.  Group g of every stream goes into one nlinv_batch call (streams
    with fewer groups drop out).
    """
    per = [groups(len(s["Y"]), s["delay"], s["warmup"]) for s in streams]
    for g in range(max(len(p) for p in per)):
        frames = []
        for s, p in zip(streams, per):
            if g >= len(p):
                continue
            for n in p[g]:
                src = source(n, s["delay"], s["warmup"])
                last = s["x"][n - 1] if (s.get("last_from_prev") and n > 0 and src != n - 1) else None
                frames.append(dict(plan=s["plan"], Y=s["Y"][n], turn=s["turns"][n],
                                   x_prev=None if src < 0 else s["x"][src], x_out=s["x"][n],
                                   img_out=None if s.get("img") is None else s["img"][n],
                                   x_last=last))
        L.nlinv_batch(frames, stream)
