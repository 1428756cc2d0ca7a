"""Reverse-mode derivative of one NLINV frame -- TEST INFRASTRUCTURE ONLY.

FP64 restatement of the backward pass through the unrolled IRGNM / CG of
Sec. 2.2 (Eqs. (2)-(5)): the loss gradient g = dL/dx^_M is carried back
through M Newton steps and K CG iterations per step, exactly as computed
(fixed iteration counts, data-dependent step lengths), to the gridded data Y
and to alpha_0 (alpha_n = alpha_0 q^n).  Each Newton step is recomputed from
its checkpoint x^_n.

Conventions: complex vectors are real vector spaces with <u, v>_R =
Re sum conj(u) v; a gradient g satisfies dL = <g, dx>_R (for torch complex
tensors this is the .grad convention, dL/dRe + i dL/dIm).

F^ is bilinear with the symmetric form B(x, d) = DF(x)[d] = U pad(c_x d_rho +
x_rho W^-1 d_c) (c_x = W^-1 x_c), so every derivative below reduces to the
oracle's DF / DFH at other linearisation points:
  A(x) p = DF(x)^H P DF(x) p + alpha p
    -> x-bar += DF(qbar)^H P DF(x) p + DF(p)^H P DF(x) qbar
  b(x) = DF(x)^H z - alpha (x - x_ref),  z = Y - P F^(x)
    -> x-bar += DF(bbar)^H z - DF(x)^H P DF(x) bbar - alpha bbar,
       Y-bar += DF(x) bbar,  alpha-bar -= <bbar, x - x_ref>_R
"""
from __future__ import annotations

import numpy as np

from .nlinv import (XVec, Params, Geometry, DF, DFH, F_hat, normal, dot, newton_rhs)


def _cg_tape(apply, b: XVec, iters: int):
    """The CG of nlinv.cg, recording what the reverse pass needs."""
    x = XVec(np.zeros_like(b.rho), np.zeros_like(b.chat))
    r = b.copy()
    p = r.copy()
    rr = dot(r, r)
    tape = dict(p=[], q=[], r=[r.copy()], rho=[rr], gamma=[], a=[], beta=[])
    for _ in range(iters):
        if rr == 0.0:
            break
        q = apply(p)
        pq = dot(p, q)
        a = rr / pq
        x = x + p.scale(a)
        r = r - q.scale(a)
        rr_new = dot(r, r)
        beta = rr_new / rr
        tape["p"].append(p)
        tape["q"].append(q)
        tape["gamma"].append(pq)
        tape["a"].append(a)
        tape["beta"].append(beta)
        tape["r"].append(r.copy())
        tape["rho"].append(rr_new)
        p = r + p.scale(beta)
        rr = rr_new
    return x, tape


def _zero_like(v: XVec) -> XVec:
    return XVec(np.zeros_like(v.rho), np.zeros_like(v.chat))


def cg_vjp(tape, xbar: XVec, apply):
    """Reverse of the recorded CG: returns (b-bar, list of q-bar_k) for the
    output adjoint xbar; the caller adds the operator-parameter terms."""
    K = len(tape["a"])
    pbar = _zero_like(xbar)          # adjoint of p_{k+1}
    rbar = _zero_like(xbar)          # adjoint of r_{k+1}
    xb = xbar.copy()                 # adjoint of x_{k+1}
    rhobar = [0.0] * (K + 1)
    qbars = [None] * K
    for k in reversed(range(K)):
        p, q, r1 = tape["p"][k], tape["q"][k], tape["r"][k + 1]
        a, beta, gamma = tape["a"][k], tape["beta"][k], tape["gamma"][k]
        rho_k, rho_k1 = tape["rho"][k], tape["rho"][k + 1]
        # p_{k+1} = r_{k+1} + beta_k p_k
        rbar = rbar + pbar
        betabar = dot(p, pbar)
        pb = pbar.scale(beta)
        # beta_k = rho_{k+1} / rho_k
        rhobar[k + 1] += betabar / rho_k
        rhobar[k] -= betabar * rho_k1 / rho_k ** 2
        # rho_{k+1} = <r_{k+1}, r_{k+1}>
        rbar = rbar + r1.scale(2.0 * rhobar[k + 1])
        # r_{k+1} = r_k - a_k q_k
        abar = -dot(q, rbar)
        qbar = rbar.scale(-a)
        # x_{k+1} = x_k + a_k p_k
        abar += dot(p, xb)
        pb = pb + xb.scale(a)
        # a_k = rho_k / gamma_k
        rhobar[k] += abar / gamma
        gammabar = -abar * rho_k / gamma ** 2
        # gamma_k = <p_k, q_k>
        pb = pb + q.scale(gammabar)
        qbar = qbar + p.scale(gammabar)
        # q_k = A p_k   (A self-adjoint)
        pb = pb + apply(qbar)
        qbars[k] = qbar
        pbar = pb                   # now the adjoint of p_k
    # p_0 = r_0 = b, rho_0 = <r_0, r_0>
    r0 = tape["r"][0]
    bbar = rbar + pbar + r0.scale(2.0 * rhobar[0])
    return bbar, qbars


def frame_vjp(Y: np.ndarray, P: np.ndarray, x_init: XVec, x_ref: XVec, geom: Geometry,
              prm: Params, gbar: XVec):
    """Gradients of L with dL/dx^_M = gbar w.r.t. Y (complex, [J,G,G]),
    alpha_0 (real), the initial value x_init and the regulariser x_ref,
    through the unrolled frame of nlinv.nlinv_frame."""
    M = prm.newton_steps
    ckpt = [x_init.copy()]
    for n in range(M):           # forward, checkpoint x^_n
        x = ckpt[-1]
        alpha = prm.alpha0 * prm.q ** n
        b = newton_rhs(x, x_ref, Y, P, alpha, geom)
        d, _ = _cg_tape(lambda v: normal(x, v, P, alpha, geom), b, prm.cg_iters)
        ckpt.append(x + d)
    Ybar = np.zeros_like(Y)
    alpha0_bar = 0.0
    xbar = gbar.copy()
    xref_bar = _zero_like(gbar)
    for n in reversed(range(M)):
        x = ckpt[n]
        alpha = prm.alpha0 * prm.q ** n
        b = newton_rhs(x, x_ref, Y, P, alpha, geom)
        A = lambda v: normal(x, v, P, alpha, geom)  # noqa: E731
        _, tape = _cg_tape(A, b, prm.cg_iters)
        bbar, qbars = cg_vjp(tape, xbar, A)
        alpha_bar = 0.0
        xb_n = xbar.copy()        # x^_{n+1} = x^_n + delta
        for p, qbar in zip(tape["p"], qbars):
            alpha_bar += dot(p, qbar)
            xb_n = xb_n + DFH(qbar, P[None] * DF(x, p, geom), geom) \
                        + DFH(p, P[None] * DF(x, qbar, geom), geom)
        z = Y - P[None] * F_hat(x, geom)
        xb_n = xb_n + DFH(bbar, z, geom) - DFH(x, P[None] * DF(x, bbar, geom), geom) \
                    - bbar.scale(alpha)
        Ybar = Ybar + DF(x, bbar, geom)
        alpha_bar -= dot(bbar, x - x_ref)
        alpha0_bar += prm.q ** n * alpha_bar
        xref_bar = xref_bar + bbar.scale(alpha)
        xbar = xb_n
    return Ybar, alpha0_bar, xbar, xref_bar
