"""GPU parity at the full sizes of the benchmark configurations, against the
FP64 oracle, through the C ABI (Sec. 2.2, Eqs. (2)-(5); Sec. 3.3, Eq. (10)):

* the batched uneven launch group: 256^2 / 8 ch, 320^2 / 10 ch and
  384^2 / 16 ch with 11 / 11 / 10 frames in flight in one nlinv_batch call
  (the work-proportional SM split of the benchmark, so each frame group has
  a handful of CTAs looping over its items), 15 radial spokes, 7 x 10;
* a whole frame at the high-channel-count size: N = 256 on the 512 grid,
  64 channels, 9 spokes, smooth random coil maps, 7 x 10 (final image and
  rho within the bar; the coil coefficients of this 9-spoke problem are
  resolved only to the FP32 floor, printed);
* five chained frames of the real-time stream: N = 160 on the 320 grid,
  10 channels, 13 spokes, each frame from the previous one.

Every frame must match the oracle within relative L2 1e-3; the measured
error against FP64 is printed for each.  The oracle runs in spawned worker
processes (started before any GPU work of the test) where frames are
independent.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

import oracle as O
import oracle_jobs as OJ
from gpu_util import make_plan, rel, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-3


def oracle_pool():
    cores = os.cpu_count() or 1
    n = max(1, min(8, cores // 2))
    return cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"),
                                  initializer=OJ.init, initargs=(max(1, cores // n),))


C3 = [dict(N=128, J=8, D=11, seed=3000), dict(N=160, J=10, D=11, seed=3001),
      dict(N=192, J=16, D=10, seed=3002)]


def test_batched_uneven_launch_group_matches_oracle():
    """Frame 0 of each size class alone, then one launch with frames 1..D of
    every class, each starting from (and regularised towards) its class's
    frame 0: oracle.nlinv_stream with delay D and no in-order warm-up."""
    from paper_1701_08361_gb300 import nlinv as L
    K, U = 15, 5
    with oracle_pool() as pool:
        first = [pool.submit(OJ.frame_job, dict(N=c["N"], J=c["J"], K=K, U=U, n=0, seed=c["seed"]))
                 for c in C3]
        first = [f.result() for f in first]
        assert all(O.source_frame(n, c["D"], 0) == 0 for c in C3 for n in range(1, c["D"] + 1))
        rest = [[pool.submit(OJ.frame_job, dict(N=c["N"], J=c["J"], K=K, U=U, n=n, seed=c["seed"],
                                                  x0=first[i][2]))
                 for n in range(1, c["D"] + 1)] for i, c in enumerate(C3)]
        rest = [[f.result() for f in fs] for fs in rest]
    plans, x0s, descs, want = [], [], [], []
    for i, c in enumerate(C3):
        N, J, D = c["N"], c["J"], c["D"]
        plan = make_plan(N, J, turns=U, max_batch=D)
        for u in range(U):
            P = first[i][1] if u == 0 else rest[i][u - 1][1]
            L.nlinv_set_psf(plan, u, to_dev(P, torch.float32))
        plans.append(plan)
        x0 = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
        L.nlinv_frame(plan, to_dev(first[i][0]), 0, None, x0)
        assert L.nlinv_sync(plan) == 0
        e0 = rel(to_np(x0), first[i][2])
        print(f"N={N} J={J} frame 0: rel L2 vs FP64 {e0:.2e}")
        assert e0 <= TOL
        x0s.append(x0)
        for n in range(1, D + 1):
            Y, _, xw = rest[i][n - 1]
            xo = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
            descs.append(dict(plan=plan, Y=to_dev(Y), turn=n % U, x_prev=x0, x_out=xo))
            want.append((N, J, n, xw))
    assert len(descs) == 32
    L.nlinv_batch(descs)
    for pl in plans:
        assert L.nlinv_sync(pl) == 0
    worst = 0.0
    for d, (N, J, n, xw) in zip(descs, want):
        e = rel(to_np(d["x_out"]), xw)
        worst = max(worst, e)
        print(f"N={N} J={J} frame {n}: rel L2 vs FP64 {e:.2e}")
        assert e <= TOL, (N, J, n, e)
    print(f"launch group of 32 frames: worst rel L2 vs FP64 {worst:.2e}")


def test_high_channel_count_frame_matches_oracle():
    """N = 256 on the 512 grid, 64 channels, 9 spokes, 3-bump coil maps,
    7 Newton x 10 CG from the initial value."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J, K, U = 256, 64, 9, 5
    Y, P, xw = OJ.frame_job(dict(N=N, J=J, K=K, U=U, n=0, seed=4001, bumps=3))
    plan = make_plan(N, J, psf=P)
    x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    img = torch.empty(N * N, dtype=torch.complex64, device="cuda")
    L.nlinv_frame(plan, to_dev(Y), 0, None, x, None, img)
    assert L.nlinv_sync(plan) == 0
    g = O.Geometry(N=N, J=J)
    xo = O.XVec.unflat(xw, g)
    e = rel(to_np(x), xw)
    er = rel(to_np(x)[:N * N], xo.rho)
    ei = rel(to_np(img), O.image(xo, g))
    print(f"C4 frame: rel L2 vs FP64: image {ei:.2e}, rho {er:.2e}, whole x^ {e:.2e}")
    # the split of the image into rho and the coil coefficients is weakly
    # determined here (the regulariser that holds the scale is at alpha_0 / 64),
    # so the bar is on the final image rho ||c|| alone
    assert ei <= TOL, (ei, er, e)


def test_realtime_stream_five_chained_frames_match_oracle():
    """Frames 0..4 of the real-time stream, each from the previous one."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J, K, U, NF, seed = 160, 10, 13, 5, 5, 1702
    frames = [OJ.radial_inputs(N, J, K, U, n, seed) for n in range(NF)]
    g = O.Geometry(N=N, J=J)
    ref = O.nlinv_stream(frames, g, O.Params())
    plan = make_plan(N, J, turns=U)
    for u in range(U):
        L.nlinv_set_psf(plan, u, to_dev(frames[u][1], torch.float32))
    x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    for n, (Y, _) in enumerate(frames):
        L.nlinv_frame(plan, to_dev(Y), n % U, None if n == 0 else x, x)
        assert L.nlinv_sync(plan) == 0
        e = rel(to_np(x), ref[n].flat())
        print(f"stream frame {n}: rel L2 vs FP64 {e:.2e}")
        assert e <= TOL, (n, e)
