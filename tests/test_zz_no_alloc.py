"""The allocation-free normal operator (nlinv_apply_normal_static).

Callers that cannot allocate device memory -- a running real-time loop that
must not call cudaMalloc, or a framework that owns all device memory -- use
this entry point; it keeps its intermediates in the library's fixed device
array.  Its result must equal the plan-based nlinv_apply_normal within the
per-application tolerance, on consecutive calls that reuse the array.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth as S
from gpu_util import geometry, make_plan, radial_psf, random_xhat, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("N,J,Gc", [(20, 3, 0), (160, 10, 0), (64, 4, 32)])
def test_static_matches_plan_entry_point_on_two_calls(N, J, Gc):
    from paper_1701_08361_gb300 import nlinv as L
    P, _, _ = radial_psf(N, 9, 5, 1)
    plan = make_plan(N, J, Gc, psf=P)
    g = geometry(plan)
    Pd = to_dev(P, torch.float32)
    for call, seed in enumerate((101, 202)):
        x, d = random_xhat(g, seed), random_xhat(g, seed + 7)
        xd, dd = to_dev(x.flat()), to_dev(d.flat())
        want = torch.empty_like(xd)
        got = torch.empty_like(xd)
        alpha = 0.25 / (call + 1)
        L.nlinv_apply_normal(plan, xd, dd, 0, alpha, want)
        L.nlinv_apply_normal_static(N, J, Gc, 220.0, 32.0, xd, dd, Pd, alpha, got)
        assert L.nlinv_sync(plan) == 0
        torch.cuda.synchronize()
        assert rel(to_np(got), to_np(want)) <= TOL, call
        # and both against the FP64 oracle
        assert rel(to_np(got), O.normal(x, d, P, alpha, g).flat()) <= TOL, call


def test_static_rejects_sizes_beyond_its_array():
    from paper_1701_08361_gb300 import nlinv as L
    N, J = 256, 8            # needs about 40 J N^2 bytes = 21 MB > 16 MiB
    G, Gc = 2 * N, N // 2
    nx = N * N + J * Gc * Gc
    x = torch.zeros(nx, dtype=torch.complex64, device="cuda")
    o = torch.zeros_like(x)
    P = torch.zeros(G * G, dtype=torch.float32, device="cuda")
    with pytest.raises(L.NlinvError) as e:
        L.nlinv_apply_normal_static(N, J, 0, 220.0, 32.0, x, x, P, 0.1, o)
    assert e.value.code == L.NLINV_EINVAL


def test_static_allocates_no_device_memory():
    """After the first call on the device (its one-time set-up), further
    calls leave the device's free memory unchanged: nothing is allocated."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J = 64, 4
    P, _, _ = radial_psf(N, 9, 5, 2)
    g = O.Geometry(N=N, J=J)
    x, d = random_xhat(g, 301), random_xhat(g, 302)
    xd, dd, Pd = to_dev(x.flat()), to_dev(d.flat()), to_dev(P, torch.float32)
    out = torch.empty_like(xd)
    L.nlinv_apply_normal_static(N, J, 0, 220.0, 32.0, xd, dd, Pd, 0.5, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for alpha in (0.5, 0.25, 0.125):
        L.nlinv_apply_normal_static(N, J, 0, 220.0, 32.0, xd, dd, Pd, alpha, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert rel(to_np(out), O.normal(x, d, P, 0.125, g).flat()) <= TOL


def test_static_tables_follow_a_change_of_sizes():
    """Calls alternating between grid sizes and weight constants: each call's
    result matches the plan entry point (the cached tables are rewritten
    whenever G, Gc, w_a or w_l change)."""
    from paper_1701_08361_gb300 import nlinv as L
    for N, J, Gc, w_a in [(20, 3, 0, 220.0), (64, 4, 32, 220.0), (20, 3, 0, 220.0), (20, 3, 0, 55.0)]:
        P, _, _ = radial_psf(N, 9, 5, 0)
        plan = make_plan(N, J, Gc, psf=P, w_a=w_a)
        g = geometry(plan)
        x, d = random_xhat(g, 400 + N), random_xhat(g, 401 + N)
        xd, dd = to_dev(x.flat()), to_dev(d.flat())
        want, got = torch.empty_like(xd), torch.empty_like(xd)
        L.nlinv_apply_normal(plan, xd, dd, 0, 0.3, want)
        L.nlinv_apply_normal_static(N, J, Gc, w_a, 32.0, xd, dd, to_dev(P, torch.float32), 0.3, got)
        assert L.nlinv_sync(plan) == 0
        torch.cuda.synchronize()
        assert rel(to_np(got), to_np(want)) <= TOL, (N, J, Gc, w_a)
