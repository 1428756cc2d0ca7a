"""GPU parity of the operator entry points against the FP64 oracle
(Sec. 2.2, Eqs. (4)-(5)): DF, DF^H, the normal operator, the PSF and the
gridding, each through the C ABI, at sizes that span several tiles and a
ragged tail, every supported grid size, and with and without the coil crop.
Tolerance: relative L2 error <= 1e-5 per application, per part."""
import numpy as np
import pytest
import torch

import oracle as O
import synth as S
from gpu_util import geometry, make_plan, radial_psf, random_xhat, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-5

# (N, J, Gc): every compiled grid G = 2N; ragged row groups / coil tiles;
# no crop (Gc = G) and non-default crops
CASES = [(8, 2, 0), (8, 3, 16), (12, 2, 0), (20, 3, 0), (20, 2, 12), (32, 4, 0),
         (64, 4, 0), (128, 3, 0), (160, 10, 0), (192, 2, 0), (256, 2, 0)]


def split_err(got, want, g):
    NN = g.N * g.N
    return rel(got[:NN], want[:NN]), rel(got[NN:], want[NN:])


@pytest.mark.parametrize("N,J,Gc", CASES)
def test_apply_DF(N, J, Gc):
    from paper_1701_08361_gb300 import nlinv as L
    plan = make_plan(N, J, Gc)
    g = geometry(plan)
    x, d = random_xhat(g, 1), random_xhat(g, 5)
    z = torch.empty(J * g.G * g.G, dtype=torch.complex64, device="cuda")
    L.nlinv_apply_DF(plan, to_dev(x.flat()), to_dev(d.flat()), z)
    assert L.nlinv_sync(plan) == 0
    want = O.DF(x, d, g)
    assert rel(to_np(z), want) <= TOL


@pytest.mark.parametrize("N,J,Gc", CASES)
def test_apply_DFH(N, J, Gc):
    from paper_1701_08361_gb300 import nlinv as L
    plan = make_plan(N, J, Gc)
    g = geometry(plan)
    x = random_xhat(g, 11)
    zz = S.random_complex((J, g.G, g.G), 12)
    out = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    L.nlinv_apply_DFH(plan, to_dev(x.flat()), to_dev(zz), out)
    assert L.nlinv_sync(plan) == 0
    e_rho, e_c = split_err(to_np(out), O.DFH(x, zz, g).flat(), g)
    assert e_rho <= TOL and e_c <= TOL, (e_rho, e_c)


@pytest.mark.parametrize("N,J,Gc", CASES)
def test_apply_normal_radial_psf(N, J, Gc):
    from paper_1701_08361_gb300 import nlinv as L
    P, _, _ = radial_psf(N, 7, 5, 3)
    plan = make_plan(N, J, Gc, turns=2)
    L.nlinv_set_psf(plan, 1, to_dev(P, torch.float32))
    g = geometry(plan)
    x, d = random_xhat(g, 21), random_xhat(g, 23)
    out = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    L.nlinv_apply_normal(plan, to_dev(x.flat()), to_dev(d.flat()), 1, 0.125, out)
    assert L.nlinv_sync(plan) == 0
    e_rho, e_c = split_err(to_np(out), O.normal(x, d, P, 0.125, g).flat(), g)
    assert e_rho <= TOL and e_c <= TOL, (e_rho, e_c)


@pytest.mark.parametrize("N,J", [(20, 3), (160, 10)])
def test_gpu_adjoint_dot_test(N, J):
    """<DF d, z> = <d, DF^H z> on the GPU at FP32 accuracy."""
    from paper_1701_08361_gb300 import nlinv as L
    plan = make_plan(N, J)
    g = geometry(plan)
    x, d = random_xhat(g, 31), random_xhat(g, 33)
    zz = S.random_complex((J, g.G, g.G), 35)
    xd, dd, zd = to_dev(x.flat()), to_dev(d.flat()), to_dev(zz)
    z = torch.empty_like(zd)
    o = torch.empty_like(dd)
    L.nlinv_apply_DF(plan, xd, dd, z)
    L.nlinv_apply_DFH(plan, xd, zd, o)
    assert L.nlinv_sync(plan) == 0
    a = np.vdot(to_np(zd), to_np(z))
    b = np.vdot(to_np(o), to_np(dd))
    assert abs(a - b) <= 1e-5 * abs(a)


@pytest.mark.parametrize("N,K", [(8, 3), (20, 5), (64, 9), (160, 13)])
def test_psf_from_trajectory(N, K):
    from paper_1701_08361_gb300 import nlinv as L
    P, kx, ky = radial_psf(N, K, 5, 2)
    plan = make_plan(N, 2, turns=3)
    kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
    Pd = torch.empty(4 * N * N, dtype=torch.float32, device="cuda")
    L.nlinv_psf(plan, 2, kxy, Pd)
    assert L.nlinv_sync(plan) == 0
    assert rel(to_np(Pd), P) <= TOL


@pytest.mark.parametrize("N,J,K", [(8, 2, 3), (20, 3, 5), (160, 10, 13)])
def test_grid_adjoint_ndft(N, J, K):
    from paper_1701_08361_gb300 import nlinv as L
    kx, ky = S.radial_trajectory(N, K, 5, 1)
    y = S.random_complex((J, len(kx)), 7)
    want = O.grid_data(kx, ky, y, N, 2 * N)
    plan = make_plan(N, J)
    kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
    Y = torch.empty(J * 4 * N * N, dtype=torch.complex64, device="cuda")
    L.nlinv_grid(plan, kxy, to_dev(y), Y)
    assert L.nlinv_sync(plan) == 0
    assert rel(to_np(Y), want) <= TOL


def test_bad_turn_and_alias_rejected():
    from paper_1701_08361_gb300 import nlinv as L
    plan = make_plan(8, 2)
    x = torch.zeros(plan.nx, dtype=torch.complex64, device="cuda")
    o = torch.zeros_like(x)
    with pytest.raises(L.NlinvError) as e:
        L.nlinv_apply_normal(plan, x, x, 1, 0.1, o)
    assert e.value.code == L.NLINV_EINVAL
    with pytest.raises(L.NlinvError):
        L.nlinv_apply_normal(plan, x, x, 0, 0.1, x)


def test_bounded_wait_reports_timeout():
    """A device wait on a flag that nothing sets gives up after its poll
    limit and the plan reports NLINV_ETIMEOUT; the context stays usable."""
    from paper_1701_08361_gb300 import nlinv as L
    plan = make_plan(8, 2)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.nlinv_wait_flag(plan, flag, 1, 1000)
    assert L.nlinv_sync(plan) == L.NLINV_ETIMEOUT
    assert L.nlinv_sync(plan) == 0
    flag.fill_(1)
    L.nlinv_wait_flag(plan, flag, 1, 1000)
    assert L.nlinv_sync(plan) == 0


@pytest.mark.slow
def test_apply_normal_C4_size():
    """The high-channel-count configuration at full size: N=256 on the 512
    grid, 64 channels (Gc = 128), radial 9-spoke PSF; the 64-channel sum of
    the adjoint and every coil column pass in one application."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J = 256, 64
    P, _, _ = radial_psf(N, 9, 5, 0)
    plan = make_plan(N, J, turns=1, psf=P)
    g = geometry(plan)
    x, d = random_xhat(g, 41), random_xhat(g, 43)
    out = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    L.nlinv_apply_normal(plan, to_dev(x.flat()), to_dev(d.flat()), 0, 0.0625, out)
    assert L.nlinv_sync(plan) == 0
    e_rho, e_c = split_err(to_np(out), O.normal(x, d, P, 0.0625, g).flat(), g)
    assert e_rho <= TOL and e_c <= TOL, (e_rho, e_c)
