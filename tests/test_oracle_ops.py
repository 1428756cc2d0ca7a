"""Pins of the oracle's forward model, derivative, adjoint and normal operator
(Sec. 2.2, Eqs. (4)-(5)) against closed forms and invariants (CPU only)."""
import os

import numpy as np
import pytest

import oracle as O
import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rand_x(g, seed, scale=1.0):
    return O.XVec(S.random_complex((g.N, g.N), seed, scale),
                  S.random_complex((g.J, g.gc, g.gc), seed + 1, scale))


# the twofold grid, and grids G = 2 gamma N of Eq. (8) with odd G and odd Gc
GEOMS = [O.Geometry(N=8, J=2), O.Geometry(N=8, J=3, Gc=16), O.Geometry(N=12, J=2),
         O.Geometry(N=10, J=4, Gc=8), O.Geometry(N=8, J=2, grid=20), O.Geometry(N=6, J=2, grid=15),
         O.Geometry(N=8, J=3, grid=24, Gc=8)]


@pytest.mark.parametrize("g", GEOMS)
def test_DF_DFH_adjoint(g):
    x, d = rand_x(g, 1), rand_x(g, 3)
    z = S.random_complex((g.J, g.G, g.G), 5)
    lhs = np.vdot(z, O.DF(x, d, g))
    rhs = np.vdot(O.DFH(x, z, g).flat(), d.flat())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("g", GEOMS)
def test_DF_is_exact_derivative_of_bilinear_F(g):
    """F^ is bilinear in (rho, c^), so F^(x + e d) - F^(x) - e DF d is exactly
    e^2 U pad(drho W^-1 dc^)."""
    x, d = rand_x(g, 7), rand_x(g, 9)
    eps = 0.37
    lhs = O.F_hat(x + d.scale(eps), g) - O.F_hat(x, g) - eps * O.DF(x, d, g)
    rhs = eps ** 2 * O.fft2u(O.pad_img(d.rho[None] * O.W_inv(d.chat, g), g.G))
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


def test_F_hat_closed_form_point_object():
    """Single coil with only the zero-frequency coefficient a: c = a/G on the
    FOV; with rho a unit spike at r0, F^(f) = a/G^2 exp(-2 pi i f.r0/G)."""
    g = O.Geometry(N=8, J=1)
    G = g.G
    x = O.XVec.zeros(g)
    a = 0.7 - 0.2j
    x.chat[0, 0, 0] = a
    r0 = (3, 5)  # (y, x)
    x.rho[r0] = 1.0
    fy, fx = np.mgrid[0:G, 0:G]
    exp = a / G ** 2 * np.exp(-2j * np.pi * (fy * r0[0] + fx * r0[1]) / G)
    np.testing.assert_allclose(O.F_hat(x, g)[0], exp, atol=1e-16)


@pytest.mark.parametrize("g", GEOMS[:3])
def test_normal_op_selfadjoint_pd(g):
    x = rand_x(g, 11)
    rng = np.random.default_rng(2)
    P = rng.uniform(0, 1, (g.G, g.G)) * (rng.uniform(size=(g.G, g.G)) < 0.4)
    u, v = rand_x(g, 13), rand_x(g, 15)
    Au, Av = O.normal(x, u, P, 0.1, g), O.normal(x, v, P, 0.1, g)
    assert abs(np.vdot(u.flat(), Av.flat()) - np.vdot(Au.flat(), v.flat())) < 1e-12 * np.linalg.norm(Au.flat()) * np.linalg.norm(v.flat())
    assert O.dot(u, Au) > 0 and O.dot(v, Av) > 0
    # equals DFH o P o DF + alpha I
    ref = O.DFH(x, P[None] * O.DF(x, u, g), g) + u.scale(0.1)
    assert np.linalg.norm((Au - ref).flat()) <= 1e-14 * np.linalg.norm(ref.flat())


def test_four_ffts_per_channel_per_iteration(monkeypatch):
    """Sec. 2.2: one application of the normal operator applies the FFT four
    times per channel (W^-1, the PSF pair, W^-H)."""
    vals = dict(l.split() for l in open(os.path.join(GOLD, "paper_fft_count.txt"))
                if l.strip() and not l.startswith("#"))
    g = O.Geometry(N=8, J=int(vals["channels"]))
    count = [0]
    f0, i0 = O.nlinv.fft2u, O.nlinv.ifft2u

    def cf(x):
        count[0] += int(np.prod(x.shape[:-2]))
        return f0(x)

    def ci(x):
        count[0] += int(np.prod(x.shape[:-2]))
        return i0(x)

    x, d = rand_x(g, 1), rand_x(g, 2)
    P = np.ones((g.G, g.G))
    c = O.coils(x, g)          # once per Newton step, not per iteration
    monkeypatch.setattr(O.nlinv, "fft2u", cf)
    monkeypatch.setattr(O.nlinv, "ifft2u", ci)
    monkeypatch.setattr(O.nlinv, "coils", lambda xx, gg: c)
    O.normal(x, d, P, 0.5, g)
    per_ch = count[0] / g.J
    assert per_ch == int(vals["ffts_per_channel_per_cg_iteration"])
    assert per_ch * g.J * int(vals["cg_iterations"]) == int(vals["ffts_per_image"])


@pytest.mark.parametrize("N,G", [(16, 32), (12, 36), (10, 30), (8, 22)])
def test_crop_of_coil_grid_is_exact_in_fp64(N, G):
    """Sec. 3.2 crop: the discarded band carries D^-1 <= (1 + 220/16)^-16, so
    the normal operator on the cropped grid equals the uncropped one
    restricted to the kept band (rel 1e-12); on the twofold grid and on
    grids G = 2 gamma N (Eq. (8)) where Gc = floor(G/4) may be odd."""
    gf = O.Geometry(N=N, J=2, Gc=G, grid=G)
    gcr = O.Geometry(N=N, J=2, grid=G)
    x = rand_x(gcr, 21)
    d = rand_x(gcr, 23)
    xf = O.XVec(x.rho, O.crop_coef(O.pad_coef(x.chat, gf.G), gf.gc))
    df = O.XVec(d.rho, O.crop_coef(O.pad_coef(d.chat, gf.G), gf.gc))
    P = (np.random.default_rng(0).uniform(size=(gf.G, gf.G)) < 0.5).astype(float)
    a = O.normal(x, d, P, 0.3, gcr)
    b = O.normal(xf, df, P, 0.3, gf)
    bc = O.XVec(b.rho, O.crop_coef(O.pad_coef(b.chat, gf.G), gcr.gc))
    assert np.linalg.norm((a - bc).flat()) <= 1e-12 * np.linalg.norm(a.flat())
