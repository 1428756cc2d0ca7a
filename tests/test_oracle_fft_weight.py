"""Pins of the oracle's grid helpers and Sobolev weight against closed forms,
brute force and the paper's printed numbers (CPU only)."""
import os

import numpy as np
import pytest

import oracle as O
import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dft_matrix(n, sign=-1):
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


@pytest.mark.parametrize("shape", [(8, 8), (3, 5), (15, 24), (24, 15)])
def test_fft2u_is_brute_force_unitary_dft(shape):
    a, b = shape
    x = S.random_complex(shape, 11)
    ref = dft_matrix(a) @ x @ dft_matrix(b).T / np.sqrt(a * b)
    assert np.max(np.abs(O.fft2u(x) - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    refi = dft_matrix(a, +1) @ x @ dft_matrix(b, +1).T / np.sqrt(a * b)
    assert np.max(np.abs(O.ifft2u(x) - refi)) <= 1e-13 * max(1.0, np.max(np.abs(refi)))


def test_fft_parseval_and_closed_forms():
    G = 16
    x = S.random_complex((G, G), 3)
    assert abs(np.linalg.norm(O.fft2u(x)) - np.linalg.norm(x)) < 1e-12
    d = np.zeros((G, G), complex)
    d[0, 0] = 1
    np.testing.assert_allclose(O.fft2u(d), np.full((G, G), 1.0 / G), atol=1e-15)
    # tone at (fy, fx) -> delta of height G at that frequency
    fy, fx = 3, 5
    yy, xx = np.mgrid[0:G, 0:G]
    tone = np.exp(2j * np.pi * (fy * yy + fx * xx) / G)
    T = O.fft2u(tone)
    exp = np.zeros((G, G), complex)
    exp[fy, fx] = G
    np.testing.assert_allclose(T, exp, atol=1e-12)


def test_freqs_and_coef_placement():
    assert list(O.freqs(8)) == [0, 1, 2, 3, -4, -3, -2, -1]
    assert list(O.freqs(5)) == [0, 1, 2, -2, -1]
    c = S.random_complex((2, 4, 4), 5)
    z = O.pad_coef(c, 16)
    # frequency f of the 4-grid lands on index f mod 16 of the 16-grid
    assert z[0, 15, 14] == c[0, 3, 2]       # f = (-1, -2)
    assert z[1, 1, 0] == c[1, 1, 0]
    assert np.count_nonzero(z) == c.size
    np.testing.assert_array_equal(O.crop_coef(z, 4), c)


def test_coil_grid_floor_rule_matches_table3():
    rows = np.loadtxt(os.path.join(GOLD, "paper_tab3_coil_grid.txt"), dtype=int)
    for N, G, gc in rows:
        assert G // 4 == gc
    # and the oracle's default for our grids (G = 2N)
    assert O.Geometry(N=160, J=10).gc == 80
    assert O.Geometry(N=64, J=4).gc == 32


def test_sobolev_weight_closed_forms():
    g = O.Geometry(N=64, J=1, Gc=128)
    D = O.sobolev_inv_weight(g)
    G = g.G
    assert D[0, 0] == 1.0
    # same as the figure's (1 + 880 |k|^2)^16 with k = f/G in (-0.5, 0.5)
    f = O.freqs(G)
    k2 = (f[:, None] / G) ** 2 + (f[None, :] / G) ** 2
    np.testing.assert_allclose(D, (1.0 + 880.0 * k2) ** -16.0, rtol=1e-14)
    # value at the edge of the G/4 crop along one axis: (1 + 220 / 16)^-16
    fx = G // 8
    assert abs(D[0, fx] - (1 + 220.0 / 16.0) ** -16) < 1e-30
    # symmetric in +-f (interior of the grid)
    for i in range(1, G // 2):
        assert D[0, i] == D[0, G - i]
        assert D[i, 0] == D[G - i, 0]


def test_W_inv_unit_coefficient_is_plane_wave():
    g = O.Geometry(N=8, J=1)
    G, Gc, N = g.G, g.gc, g.N
    D = O.sobolev_inv_weight(g)
    for (iy, ix) in [(0, 0), (1, 0), (0, 3), (3, 2)]:
        c = np.zeros((1, Gc, Gc), complex)
        c[0, iy, ix] = 1.0
        fy, fx = O.freqs(Gc)[iy], O.freqs(Gc)[ix]
        yy, xx = np.mgrid[0:N, 0:N]
        exp = D[iy, ix] * np.exp(2j * np.pi * (fx * xx + fy * yy) / G) / G
        np.testing.assert_allclose(O.W_inv(c, g)[0], exp, atol=1e-15)


@pytest.mark.parametrize("N,J,Gc", [(8, 2, None), (8, 2, 16), (12, 3, None), (10, 1, 6)])
def test_W_inv_adjoint(N, J, Gc):
    g = O.Geometry(N=N, J=J, Gc=Gc)
    a = S.random_complex((J, g.gc, g.gc), 1)
    b = S.random_complex((J, N, N), 2)
    lhs = np.vdot(b, O.W_inv(a, g))
    rhs = np.vdot(O.W_invH(b, g), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
