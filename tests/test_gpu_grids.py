"""GPU parity on grids G = 2 gamma N of Eq. (8) with gamma > 1 (the grid
sizes of Sec. 3.2 / Tab. 2 chosen for FFT speed), against the FP64 oracle
through the C ABI: the operators (relative L2 1e-5 per application, per
part), the PSF and the gridding of a radial trajectory on such a grid, and
whole frames (1e-3).  The grids use radix-3, -5 and -7 splits, odd coil grids
(Gc = floor(G/4)) and fields of view that do not fill half the grid."""
import numpy as np
import pytest
import torch

import oracle as O
import synth as S
from gpu_util import geometry, make_plan, radial_psf, random_xhat, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-5

# (N, J, G): radix 7 (56 = 4 x 14, 448 = 16 x 28, 560 = 20 x 28), radix 3^k
# (54 = 6 x 9, 72 = 8 x 9, 486 = 18 x 27), radix 3 x 5 (480 = 16 x 30), and
# gamma = 1.5 / 1.6 on power-of-two splits (384 for N = 128, 512 for N = 160)
GRIDS = [(20, 3, 56), (20, 2, 54), (24, 3, 72), (160, 4, 448), (160, 4, 480), (160, 3, 486),
         (160, 4, 512), (160, 2, 560), (128, 3, 384)]


def split_err(got, want, g):
    NN = g.N * g.N
    return rel(got[:NN], want[:NN]), rel(got[NN:], want[NN:])


@pytest.mark.parametrize("N,J,G", GRIDS)
def test_operators_on_gamma_grids(N, J, G):
    from paper_1701_08361_gb300 import nlinv as L
    P, _, _ = radial_psf(N, 7, 5, 2, G)
    plan = make_plan(N, J, psf=P, G=G)
    g = geometry(plan)
    assert g.G == G and g.gc == G // 4
    x, d = random_xhat(g, 61), random_xhat(g, 63)
    xd, dd = to_dev(x.flat()), to_dev(d.flat())
    z = torch.empty(J * G * G, dtype=torch.complex64, device="cuda")
    L.nlinv_apply_DF(plan, xd, dd, z)
    zz = S.random_complex((J, G, G), 65)
    o1 = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    L.nlinv_apply_DFH(plan, xd, to_dev(zz), o1)
    o2 = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    L.nlinv_apply_normal(plan, xd, dd, 0, 0.25, o2)
    assert L.nlinv_sync(plan) == 0
    assert rel(to_np(z), O.DF(x, d, g)) <= TOL
    for got, want in ((o1, O.DFH(x, zz, g)), (o2, O.normal(x, d, P, 0.25, g))):
        e_rho, e_c = split_err(to_np(got), want.flat(), g)
        assert e_rho <= TOL and e_c <= TOL, (e_rho, e_c)


@pytest.mark.parametrize("N,J,G", [(20, 2, 54), (24, 3, 72), (160, 3, 486)])
def test_psf_and_gridding_on_gamma_grids(N, J, G):
    from paper_1701_08361_gb300 import nlinv as L
    kx, ky = S.radial_trajectory(N, 9, 5, 3)
    y = S.random_complex((J, len(kx)), 71)
    plan = make_plan(N, J, G=G)
    kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
    Pd = torch.empty(G * G, dtype=torch.float32, device="cuda")
    L.nlinv_psf(plan, 0, kxy, Pd)
    Yd = torch.empty(J * G * G, dtype=torch.complex64, device="cuda")
    L.nlinv_grid(plan, kxy, to_dev(y), Yd)
    assert L.nlinv_sync(plan) == 0
    assert rel(to_np(Pd), O.psf_kernel(kx, ky, N, G).real) <= TOL
    assert rel(to_np(Yd), O.grid_data(kx, ky, y, N, G)) <= TOL


@pytest.mark.parametrize("N,J,G,M,K,mode", [(20, 3, 56, 3, 5, 2), (24, 3, 72, 3, 5, 1),
                                           (20, 2, 54, 3, 5, 0), (160, 10, 480, 7, 10, 0)])
def test_frames_on_gamma_grids(N, J, G, M, K, mode):
    """Radial frames (13 spokes) from the initial value on a grid with
    gamma > 1, the samples gridded by the oracle on that grid."""
    from paper_1701_08361_gb300 import nlinv as L
    g = O.Geometry(N=N, J=J, grid=G)
    kx, ky, y, _, _ = S.radial_frame(N, J, 13, 5, 2, seed=81)
    Y = O.grid_data(kx, ky, y, N, G)
    P = O.psf_kernel(kx, ky, N, G).real
    prm = O.Params(newton_steps=M, cg_iters=K)
    ref = O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g, prm)
    plan = make_plan(N, J, psf=P, G=G, newton_steps=M, cg_iters=K, exec_mode=mode)
    x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    img = torch.empty(N * N, dtype=torch.complex64, device="cuda")
    L.nlinv_frame(plan, to_dev(Y), 0, None, x, None, img)
    assert L.nlinv_sync(plan) == 0
    e, ei = rel(to_np(x), ref.flat()), rel(to_np(img), O.image(ref, g))
    print(f"N={N} G={G} J={J}: rel L2 vs FP64 x^ {e:.2e}, image {ei:.2e}")
    assert e <= 1e-3 and ei <= 1e-3


def test_grid_choices_outside_the_compiled_set_are_refused():
    from paper_1701_08361_gb300 import nlinv as L
    for N, G, code in ((160, 500, L.NLINV_EUNSUPPORTED), (160, 300, L.NLINV_EINVAL),
                       (20, 50, L.NLINV_EUNSUPPORTED)):
        with pytest.raises(L.NlinvError) as e:
            make_plan(N, 2, G=G)
        assert e.value.code == code


@pytest.mark.parametrize("N,J,G,W", [(20, 3, 40, 6), (32, 2, 64, 8), (20, 2, 54, 6), (160, 4, 320, 6),
                                     (160, 3, 486, 7)])
def test_convolution_gridding_matches_oracle(N, J, G, W):
    """nlinv_grid_nufft against the oracle's Kaiser-Bessel gridding (the same
    algorithm, 1e-5) and against the exact adjoint NDFT within the kernel
    bound (2e-5 at W >= 6)."""
    from paper_1701_08361_gb300 import nlinv as L
    kx, ky = S.radial_trajectory(N, 11, 5, 2)
    y = S.random_complex((J, len(kx)), 91)
    plan = make_plan(N, J, G=G)
    kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
    Yd = torch.empty(J * G * G, dtype=torch.complex64, device="cuda")
    L.nlinv_grid_nufft(plan, kxy, to_dev(y), W, Yd)
    assert L.nlinv_sync(plan) == 0
    got = to_np(Yd)
    e_kb = rel(got, O.grid_data_kb(kx, ky, y, N, G, W))
    e_ex = rel(got, O.grid_data(kx, ky, y, N, G))
    print(f"N={N} G={G} W={W}: vs oracle KB gridding {e_kb:.2e}, vs exact NDFT {e_ex:.2e}")
    assert e_kb <= TOL and e_ex <= 2e-5


def test_autotuner_record_and_pick():
    """The tuner times every candidate (compiled grids in the gamma range x
    execution paths), keeps the fastest, and a plan made from its record
    reconstructs the frame like the oracle on the picked grid."""
    import json
    import os
    import tempfile
    from paper_1701_08361_gb300 import nlinv as L
    from paper_1701_08361_gb300 import tune as T
    N, J, M, K = 20, 3, 2, 3
    with tempfile.TemporaryDirectory() as d:
        db = os.path.join(d, "db.json")
        rec = T.tune(N, J, M, K, gamma=(1.0, 1.5), db=db, frames=3)
        grids = {c["G"] for c in rec["candidates"]}
        assert grids == {G for G, n in L.nlinv_grid_list() if n == N and G <= 60}
        assert rec["ms_per_frame"] == min(c["ms_per_frame"] for c in rec["candidates"])
        assert {2, 4} <= {c["exec_mode"] for c in rec["candidates"]}
        assert json.load(open(db))[T.gpu_name()]
        p = T.tuned_params(N, J, M, K, gamma=(1.0, 1.5), db=db)
        assert (p.G, p.exec_mode, p.cluster_cs) == (rec["pick"]["G"], rec["pick"]["exec_mode"],
                                                     rec["pick"]["cluster_cs"])
    G = p.G
    g = O.Geometry(N=N, J=J, grid=G)
    kx, ky, y, _, _ = S.radial_frame(N, J, 13, 5, 0, seed=3)
    Y, P = O.grid_data(kx, ky, y, N, G), O.psf_kernel(kx, ky, N, G).real
    ref = O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g, O.Params(newton_steps=M, cg_iters=K))
    plan = L.nlinv_plan(p, to_dev(P, torch.float32))
    x = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    L.nlinv_frame(plan, to_dev(Y), 0, None, x)
    assert L.nlinv_sync(plan) == 0
    assert rel(to_np(x), ref.flat()) <= 1e-3


@pytest.mark.parametrize("T,n", [(1, 1000), (3, 25600), (5, 65536), (15, 777)])
def test_temporal_median_matches_oracle(T, n):
    """nlinv_median (post-processing, Sec. 3.1) against the oracle's
    pixel-wise median of the magnitudes, on images with outlier frames."""
    from paper_1701_08361_gb300 import nlinv as L
    imgs = S.random_complex((T, n), 500 + T)
    imgs[T // 2, ::7] *= 50.0                 # outliers the median must reject
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    L.nlinv_median([to_dev(imgs[t]) for t in range(T)], out)
    torch.cuda.synchronize()
    want = O.temporal_median(imgs.astype(np.complex64).astype(np.complex128))
    assert np.max(np.abs(to_np(out) - want) / np.maximum(want, 1e-30)) <= 1e-6


def test_temporal_median_rejects_even_or_long_windows():
    from paper_1701_08361_gb300 import nlinv as L
    a = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    for T in (2, 17):
        with pytest.raises(L.NlinvError):
            L.nlinv_median([a] * T, out)
