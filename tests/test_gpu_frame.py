"""GPU parity of whole NLINV frames (IRGNM + CG, Eqs. (2)-(3)) against the
FP64 oracle through the C ABI: final x^, rho and the coil-combined image
within relative L2 1e-3 (FP32 arithmetic against FP64 through 7 x 10
Newton/CG steps), in every execution mode (per-phase launches, the grid
kernel, the cluster kernel, and the automatic choice)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth as S
from gpu_util import make_plan, radial_psf, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-3


def run_frames(plan, frames, xprev=None):
    """frames: list of (Y, turn); returns list of (x, rho, img) numpy."""
    from paper_1701_08361_gb300 import nlinv as L
    N = plan.N
    x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    if xprev is not None:
        x.copy_(to_dev(xprev))
    out = []
    first = xprev is None
    for Y, turn in frames:
        rho = torch.empty(N * N, dtype=torch.complex64, device="cuda")
        img = torch.empty(N * N, dtype=torch.complex64, device="cuda")
        L.nlinv_frame(plan, to_dev(Y), turn, None if first else x, x, rho, img)
        rc = L.nlinv_sync(plan)
        assert rc == 0, L.nlinv_strerror(rc)
        out.append((to_np(x), to_np(rho), to_np(img)))
        first = False
    return out


@pytest.mark.parametrize("exec_mode", [0, 1, 2, 3, 4])
def test_cartesian_frame_C1(exec_mode):
    """64x64 image on the 128 grid, 4 coils, every 3rd line + 16 centre
    lines, sigma = 1e-3, 7 Newton x 10 CG, alpha0 = 1, q = 1/2."""
    N, J = 64, 4
    Y, P, _, _ = S.cartesian_frame(N, J, seed=1701, sigma=1e-3)
    g = O.Geometry(N=N, J=J)
    ref = O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g, O.Params())
    plan = make_plan(N, J, psf=P, exec_mode=exec_mode)
    (x, rho, img), = run_frames(plan, [(Y, 0)])
    assert rel(x, ref.flat()) <= TOL
    assert rel(rho, ref.rho) <= TOL
    assert rel(img, O.image(ref, g)) <= TOL


def test_radial_stream_with_device_psf_and_gridding():
    """Radial frames (K=13 spokes, U=5 turns) whose PSFs and gridded data are
    computed by the library from the trajectory and raw samples; 3 frames
    chained with damping 0.9."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J, K, U = 64, 4, 13, 5
    g = O.Geometry(N=N, J=J)
    prm = O.Params(damping=0.9)
    plan = make_plan(N, J, turns=U, damping=0.9)
    frames_o, frames_g = [], []
    for n in range(3):
        kx, ky, y, _, _ = S.radial_frame(N, J, K, U, n, seed=5)
        frames_o.append((O.grid_data(kx, ky, y, N, g.G), O.psf_kernel(kx, ky, N, g.G).real))
        kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
        L.nlinv_psf(plan, n % U, kxy)
        Yd = torch.empty(J * g.G * g.G, dtype=torch.complex64, device="cuda")
        L.nlinv_grid(plan, kxy, to_dev(y), Yd)
        frames_g.append((to_np(Yd), n % U))
    ref = O.nlinv_stream(frames_o, g, prm)
    got = run_frames(plan, frames_g)
    for n in range(3):
        assert rel(got[n][0], ref[n].flat()) <= TOL, n
        assert rel(got[n][2], O.image(ref[n], g)) <= TOL, n


def test_frame_from_given_x_prev_and_modes_agree():
    N, J = 20, 3
    g = O.Geometry(N=N, J=J)
    Y, P, _, _ = S.cartesian_frame(N, J, seed=9, sigma=1e-3, every=2, centre=8)
    xp = O.XVec(S.random_complex((N, N), 3, 0.5) + 1.0,
                S.random_complex((J, g.gc, g.gc), 4, 5.0))
    prm = O.Params(newton_steps=4, cg_iters=6, alpha0=2.0, q=0.6, damping=0.8)
    ref = O.nlinv_frame(Y, P, xp, xp.scale(0.8), g, prm)
    outs = []
    for mode in (1, 2, 3, 4):
        plan = make_plan(N, J, psf=P, newton_steps=4, cg_iters=6, alpha0=2.0, q=0.6,
                         damping=0.8, exec_mode=mode)
        (x, _, _), = run_frames(plan, [(Y, 0)], xprev=xp.flat())
        assert rel(x, ref.flat()) <= TOL
        outs.append(x)
    # the same arithmetic up to the order of the inner products' partial sums
    assert rel(outs[0], outs[1]) <= 1e-5
    assert rel(outs[2], outs[1]) <= 1e-5
    # the graph replays exactly the per-phase launches
    assert np.array_equal(outs[3], outs[0])


@pytest.mark.slow
def test_radial_frame_C2_size():
    """One frame at the real-time stream size: N=160 on the 320 grid, 10
    channels, 13 spokes, 7 Newton x 10 CG, preprocessing on the device."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J, K, U = 160, 10, 13, 5
    g = O.Geometry(N=N, J=J)
    kx, ky, y, _, _ = S.radial_frame(N, J, K, U, 0, seed=1702)
    Yo = O.grid_data(kx, ky, y, N, g.G)
    Po = O.psf_kernel(kx, ky, N, g.G).real
    ref = O.nlinv_frame(Yo, Po, O.XVec.initial(g), O.XVec.initial(g), g, O.Params())
    plan = make_plan(N, J, turns=U)
    kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
    L.nlinv_psf(plan, 0, kxy)
    Yd = torch.empty(J * g.G * g.G, dtype=torch.complex64, device="cuda")
    L.nlinv_grid(plan, kxy, to_dev(y), Yd)
    (x, rho, img), = run_frames(plan, [(to_np(Yd), 0)])
    assert rel(x, ref.flat()) <= TOL
    assert rel(img, O.image(ref, g)) <= TOL


@pytest.mark.slow
def test_frame_C4_size_modes_agree():
    """A whole frame at the high-channel-count size (N=256 / 512 grid, 64
    channels, 9 spokes, 7 x 10): the persistent launch and the one-launch-
    per-phase path (separate kernels, same arithmetic) agree, and the output
    is finite.  (The FP64 oracle needs minutes per frame at this size; its
    parity is checked per operator application in test_gpu_ops.)"""
    from paper_1701_08361_gb300 import nlinv as L
    N, J, K, U = 256, 64, 9, 5
    g = O.Geometry(N=N, J=J)
    kx, ky = S.radial_trajectory(N, K, U, 0)
    xs = []
    for mode in (0, 1):
        plan = make_plan(N, J, turns=1, exec_mode=mode)
        kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
        L.nlinv_psf(plan, 0, kxy)
        Yd = to_dev(S.random_complex((J, g.G, g.G), 77) * 1e-2)
        x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
        L.nlinv_frame(plan, Yd, 0, None, x)
        assert L.nlinv_sync(plan) == 0
        xs.append(to_np(x))
    assert np.all(np.isfinite(xs[0]))
    assert rel(xs[0], xs[1]) <= 1e-5


@pytest.mark.parametrize("M,K,mode", [(1, 1, 2), (1, 0, 2), (2, 1, 1), (1, 3, 1), (3, 0, 1),
                                      (1, 1, 3), (1, 0, 3), (2, 2, 3), (1, 0, 4), (2, 2, 4)])
def test_degenerate_iteration_counts(M, K, mode):
    """One Newton step, one CG iteration, or none (x^ stays the initial value):
    the drivers' edge cases against the oracle, ragged N=20 grid."""
    N, J = 20, 3
    g = O.Geometry(N=N, J=J)
    Y, P, _, _ = S.cartesian_frame(N, J, seed=61, sigma=1e-3)
    prm = O.Params(newton_steps=M, cg_iters=K)
    ref = O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g, prm)
    plan = make_plan(N, J, psf=P, newton_steps=M, cg_iters=K, exec_mode=mode)
    (x, rho, img), = run_frames(plan, [(Y, 0)])
    if K == 0:
        np.testing.assert_array_equal(x, O.XVec.initial(g).flat().astype(np.complex64))
    assert rel(x, ref.flat()) <= TOL


@pytest.mark.parametrize("N,J,M,K", [(20, 2, 1, 8), (20, 2, 5, 8), (32, 3, 2, 8)])
@pytest.mark.parametrize("exec_mode", [0, 1])
def test_cg_reaching_the_rounding_floor_is_not_a_breakdown(N, J, M, K, exec_mode):
    """Small Cartesian frames whose CG converges to the FP32 rounding floor
    within a few iterations: the per-phase path's CG (the operator applied to
    the residual) stops there instead of reporting a breakdown, and the frame
    still matches the oracle."""
    from paper_1701_08361_gb300 import nlinv as L
    Y, P = S.cartesian_frame(N, J, seed=100, sigma=1e-3, frame=0)[:2]
    g = O.Geometry(N=N, J=J)
    plan = make_plan(N, J, psf=P, newton_steps=M, cg_iters=K, exec_mode=exec_mode)
    x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    L.nlinv_frame(plan, to_dev(Y), 0, None, x)
    assert L.nlinv_sync(plan) == 0
    ref = O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g, O.Params(newton_steps=M, cg_iters=K))
    e = rel(to_np(x), ref.flat())
    print(f"N={N} J={J} M={M} K={K} mode={exec_mode}: rel L2 vs FP64 {e:.2e}")
    assert e <= TOL


@pytest.mark.parametrize("N,J,Gc,cs", [(160, 10, 0, 0), (64, 4, 0, 0), (20, 3, 0, 0), (32, 4, 16, 0),
                                       (128, 8, 0, 8), (128, 8, 0, 0), (64, 4, 0, 6)])
def test_cluster_kernel_matches_oracle_and_grid_kernel(N, J, Gc, cs):
    """The cluster-resident frame kernel (one cluster per channel; ragged
    partitions of rows, columns and coil columns for most sizes) against the
    FP64 oracle and against the grid kernel, on a radial frame from the
    initial value (3 Newton x 5 CG)."""
    from paper_1701_08361_gb300 import nlinv as L
    K, U = 13, 5
    P, kx, ky = radial_psf(N, K, U, 1)
    g = O.Geometry(N=N, J=J, Gc=Gc or None)
    coils = S.coil_maps(N, J, 7)
    _, _, y, _, _ = S.radial_frame(N, J, K, U, 1, seed=7, coils=coils)
    Y = O.grid_data(kx, ky, y, N, g.G)
    prm = O.Params(newton_steps=3, cg_iters=5)
    ref = O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g, prm)
    xs = []
    for mode in (3, 2):
        plan = make_plan(N, J, Gc, psf=P, newton_steps=3, cg_iters=5, exec_mode=mode,
                         cluster_cs=cs if mode == 3 else 0)
        if mode == 3:
            assert L.nlinv_plan_path(plan)[0] == 3 and (cs == 0 or L.nlinv_plan_path(plan)[1] == cs)
        (x, rho, img), = run_frames(plan, [(Y, 0)])
        e = rel(x, ref.flat())
        print(f"N={N} J={J} mode {mode}: rel L2 vs FP64 {e:.2e}")
        assert e <= TOL
        xs.append(x)
    assert rel(xs[0], xs[1]) <= 1e-4


def test_graph_path_replays_over_a_stream_and_follows_alpha0():
    """exec_mode 4: the captured per-phase frame replayed for a chained
    radial stream (different data, turns and x_prev per frame, outputs only
    where asked) equals the per-phase launches bit for bit, and a change of
    alpha_0 re-captures the graph."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J, K, U = 32, 3, 13, 5
    frames, Ps = [], []
    coils = S.coil_maps(N, J, 4)
    for n in range(4):
        kx, ky, y, _, _ = S.radial_frame(N, J, K, U, n, seed=4, coils=coils)
        frames.append(O.grid_data(kx, ky, y, N, 2 * N))
        Ps.append(O.psf_kernel(kx, ky, N, 2 * N).real)
    outs = {}
    for mode in (1, 4):
        plan = make_plan(N, J, turns=U, exec_mode=mode, newton_steps=3, cg_iters=4)
        for u in range(4):
            L.nlinv_set_psf(plan, u, to_dev(Ps[u], torch.float32))
        x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
        res = []
        for n, Y in enumerate(frames):
            if n == 2:
                L.nlinv_set_alpha0(plan, 0.5)
            img = torch.zeros(N * N, dtype=torch.complex64, device="cuda") if n % 2 else None
            L.nlinv_frame(plan, to_dev(Y), n, None if n == 0 else x, x, None, img)
            assert L.nlinv_sync(plan) == 0
            res.append((to_np(x), None if img is None else to_np(img)))
        outs[mode] = res
    for (a, ia), (b, ib) in zip(outs[1], outs[4]):
        assert np.array_equal(a, b)
        assert (ia is None and ib is None) or np.array_equal(ia, ib)
