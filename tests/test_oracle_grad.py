"""Pins of the oracle's reverse-mode frame derivative (oracle/grad.py) against
FP64 central finite differences of the forward oracle (CPU only)."""
import numpy as np
import pytest

import oracle as O
from oracle import grad as OG
import synth as S


def rand_x(g, seed, scale=1.0):
    return O.XVec(S.random_complex((g.N, g.N), seed, scale),
                  S.random_complex((g.J, g.gc, g.gc), seed + 1, scale))


def setup(N=8, J=2, seed=3):
    g = O.Geometry(N=N, J=J)
    Y, P, _, _ = S.cartesian_frame(N, J, seed=seed, sigma=1e-3, every=2, centre=4)
    x0 = O.XVec(S.random_complex((N, N), 70, 0.2) + 1.0, S.random_complex((J, g.gc, g.gc), 71, 10.0))
    return g, Y, P, x0


def loss(Y, P, x0, g, prm, gvec):
    return O.dot(gvec, O.nlinv_frame(Y, P, x0, x0.scale(prm.damping), g, prm))


@pytest.mark.parametrize("M,K", [(1, 1), (2, 3), (3, 5)])
def test_frame_gradients_match_central_differences(M, K):
    g, Y, P, x0 = setup()
    prm = O.Params(newton_steps=M, cg_iters=K, alpha0=1.0, q=0.5, damping=0.9)
    gvec = rand_x(g, 90)
    Ybar, a0bar, xbar, xrbar = OG.frame_vjp(Y, P, x0, x0.scale(0.9), g, prm, gvec)
    # alpha_0
    h = 1e-5
    lp = loss(Y, P, x0, g, O.Params(M, K, 1.0 + h, 0.5, 0.9), gvec)
    lm = loss(Y, P, x0, g, O.Params(M, K, 1.0 - h, 0.5, 0.9), gvec)
    fd = (lp - lm) / (2 * h)
    assert abs(a0bar - fd) <= 1e-6 * max(abs(fd), 1e-12) + 1e-9, (a0bar, fd)
    # Y along a random complex direction
    dY = S.random_complex(Y.shape, 91)
    h = 1e-6
    fd = (loss(Y + h * dY, P, x0, g, prm, gvec) - loss(Y - h * dY, P, x0, g, prm, gvec)) / (2 * h)
    an = float(np.real(np.vdot(Ybar, dY)))
    assert abs(an - fd) <= 1e-6 * abs(fd), (an, fd)
    # x_prev (initial value and regulariser x_ref = 0.9 x_prev) along a direction
    dx = rand_x(g, 92)
    fd = (loss(Y, P, x0 + dx.scale(h), g, prm, gvec) - loss(Y, P, x0 - dx.scale(h), g, prm, gvec)) / (2 * h)
    an = O.dot(xbar + xrbar.scale(0.9), dx)
    assert abs(an - fd) <= 1e-6 * abs(fd), (an, fd)


def test_operator_linearisation_point_vjp():
    """d/dx <qbar, A(x) p>_R = DF(qbar)^H P DF(x) p + DF(p)^H P DF(x) qbar."""
    g, _, P, _ = setup()
    x, p, qbar, e = rand_x(g, 1, 1.0), rand_x(g, 2), rand_x(g, 3), rand_x(g, 4)
    x.chat *= 10
    an = O.DFH(qbar, P[None] * O.DF(x, p, g), g) + O.DFH(p, P[None] * O.DF(x, qbar, g), g)
    h = 1e-6
    fd = (O.dot(qbar, O.normal(x + e.scale(h), p, P, 0.3, g)) -
          O.dot(qbar, O.normal(x - e.scale(h), p, P, 0.3, g))) / (2 * h)
    assert abs(O.dot(an, e) - fd) <= 1e-7 * abs(fd)


def test_rhs_linearisation_point_vjp():
    """d/dx <bbar, b(x)>_R = DF(bbar)^H z - DF(x)^H P DF(x) bbar - alpha bbar."""
    g, Y, P, _ = setup()
    x, xr, bbar, e = rand_x(g, 11), rand_x(g, 12), rand_x(g, 13), rand_x(g, 14)
    x.chat *= 10
    alpha = 0.7
    z = Y - P[None] * O.F_hat(x, g)
    an = O.DFH(bbar, z, g) - O.DFH(x, P[None] * O.DF(x, bbar, g), g) - bbar.scale(alpha)
    h = 1e-6
    fd = (O.dot(bbar, O.newton_rhs(x + e.scale(h), xr, Y, P, alpha, g)) -
          O.dot(bbar, O.newton_rhs(x - e.scale(h), xr, Y, P, alpha, g))) / (2 * h)
    assert abs(O.dot(an, e) - fd) <= 1e-7 * abs(fd)
