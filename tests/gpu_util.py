"""Helpers shared by the GPU parity tests: numpy <-> device conversion, plan
construction, error measures.  No arithmetic of the method lives here."""
import numpy as np
import torch

import oracle as O
import synth as S


def dev():
    return torch.device("cuda:0")


def to_dev(a, dtype=torch.complex64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev())


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_plan(N, J, Gc=0, turns=1, psf=None, **kw):
    from paper_1701_08361_gb300 import nlinv as L
    p = L.nlinv_default_params(N, J)
    p.Gc = Gc
    p.n_turns = turns
    for k, v in kw.items():
        setattr(p, k, v)
    return L.nlinv_plan(p, None if psf is None else to_dev(psf, torch.float32))


def geometry(plan):
    return O.Geometry(N=plan.N, J=plan.J, Gc=plan.Gc, grid=plan.G)


def random_xhat(g, seed, coil_scale=None):
    """x^ with an O(1) image and coil coefficients large enough that the
    coil maps W^-1 c^ are O(1) in the FOV."""
    cs = g.G if coil_scale is None else coil_scale
    return O.XVec(S.random_complex((g.N, g.N), seed),
                  S.random_complex((g.J, g.gc, g.gc), seed + 1, cs))


def radial_psf(N, K, U, turn, G=None):
    kx, ky = S.radial_trajectory(N, K, U, turn)
    return O.psf_kernel(kx, ky, N, G or 2 * N).real, kx, ky
