"""The GPU's per-phase path runs each Newton step's CG in the arrangement of
Chronopoulos and Gear (the operator applied to the residual, both inner
products from one pass, s_k = A p_k carried by a recurrence), the oracle runs
the textbook CG of Sec. 2.2.  These CPU tests restate the Chronopoulos-Gear
recurrences from their published definition and check that they produce the
oracle's iterate (the same Krylov iterate in exact arithmetic), on a random
SPD matrix and on the oracle's own NLINV normal operator, and that its
rounding-floor stop (a = 0 once gamma_k <= 1e-8 gamma_0 and the denominator
is not positive) changes the result only at that floor."""
import numpy as np
import pytest

import oracle as O
import synth as S


def cg_residual_form(apply, b, iters, dot, axpy, floor=1e-8, perturb=None):
    """x after `iters` CG steps from zero in the Chronopoulos-Gear form:
    w_k = A r_k; gamma_k = <r_k, r_k>, delta_k = Re<r_k, w_k>;
    beta_k = gamma_k / gamma_{k-1}; a_k = gamma_k / (delta_k - beta_k gamma_k / a_{k-1});
    p_k = r_k + beta_k p_{k-1}; s_k = w_k + beta_k s_{k-1};
    x += a_k p_k; r_{k+1} = r_k - a_k s_k.  `perturb(k, den)` may replace the
    denominator (to exercise the stop rule)."""
    r = b
    x = p = s = None
    g_prev = a_prev = None
    g0 = None
    stopped = False
    for k in range(iters):
        w = apply(r)
        g, d = dot(r, r), dot(r, w)
        g0 = g if g0 is None else g0
        beta = 0.0 if k == 0 or g_prev == 0.0 else g / g_prev
        den = d if k == 0 or a_prev == 0.0 else d - beta * g / a_prev
        if perturb is not None:
            den = perturb(k, den)
        if stopped or g == 0.0:
            a = 0.0
        elif den > 0.0 and np.isfinite(den):
            a = g / den
        elif g <= floor * g0:
            a, stopped = 0.0, True
        else:
            raise O.CGBreakdown(f"denominator {den}")
        if stopped:
            beta = 0.0
        p = r if k == 0 else axpy(beta, p, r)
        s = w if k == 0 else axpy(beta, s, w)
        x = axpy(a, p, None) if x is None else axpy(a, p, x)
        r = axpy(-a, s, r)
        g_prev, a_prev = g, a
    return x


def _np_ops():
    dot = lambda u, v: float(np.real(np.vdot(u, v)))
    axpy = lambda a, u, v: a * u if v is None else a * u + v
    return dot, axpy


@pytest.mark.parametrize("n,iters,seed", [(40, 5, 1), (60, 12, 2), (25, 25, 3)])
def test_residual_form_equals_textbook_cg_on_spd_matrices(n, iters, seed):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = Q.conj().T @ Q / n + 0.3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    dot, axpy = _np_ops()
    x_cgr = cg_residual_form(lambda v: A @ v, b, iters, dot, axpy)
    # textbook CG through the oracle, the vector stored as the rho part
    g = O.Geometry(N=1, J=1, Gc=1)
    as_x = lambda v: O.XVec(v.reshape(n, 1), np.zeros((1, 1, 1), complex))
    x_ref = O.cg(lambda xv: as_x(A @ xv.rho.ravel()), as_x(b), iters)
    # both arrangements round differently; a wrong recurrence misses by orders of magnitude
    assert np.linalg.norm(x_cgr - x_ref.rho.ravel()) <= 1e-9 * np.linalg.norm(x_ref.rho)
    if iters >= n:   # a full-length CG solves the system
        assert np.linalg.norm(A @ x_cgr - b) <= 1e-6 * np.linalg.norm(b)   # finite-precision CG: ~5e-8


def test_residual_form_equals_oracle_cg_on_the_nlinv_normal_operator():
    """One Newton step's CG (7 x 10 at N = 16, 3 channels, radial PSF) in both
    arrangements, at a non-trivial linearisation point."""
    N, J = 16, 3
    g = O.Geometry(N=N, J=J)
    kx, ky, y, _, _ = S.radial_frame(N, J, 11, 5, 0, seed=7)
    Y, P = O.grid_data(kx, ky, y, N, g.G), O.psf_kernel(kx, ky, N, g.G).real
    x = O.XVec(S.random_complex((N, N), 3, 0.3) + 1.0, S.random_complex((J, g.gc, g.gc), 4, 2.0))
    alpha = 0.25
    apply = lambda d: O.normal(x, d, P, alpha, g)
    b = O.newton_rhs(x, x.scale(0.9), Y, P, alpha, g)
    x_ref = O.cg(apply, b, 10)
    dot = O.dot
    axpy = lambda a, u, v: u.scale(a) if v is None else u.scale(a) + v
    x_cgr = cg_residual_form(apply, b, 10, dot, axpy)
    d = x_cgr - x_ref
    assert np.sqrt(dot(d, d)) <= 1e-10 * np.sqrt(dot(x_ref, x_ref))


def test_rounding_floor_stop_only_acts_at_the_floor():
    rng = np.random.default_rng(5)
    n = 30
    U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    A = U @ np.diag(np.repeat([1.0, 4.0], n // 2)) @ U.conj().T   # two eigenvalues: converges in 2 steps
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    dot, axpy = _np_ops()
    x_exact = np.linalg.solve(A, b)
    # a non-positive denominator after convergence (gamma at the floor): stop, same solution
    x_stop = cg_residual_form(lambda v: A @ v, b, 6, dot, axpy, perturb=lambda k, den: -1.0 if k >= 3 else den)
    assert np.linalg.norm(x_stop - x_exact) <= 1e-10 * np.linalg.norm(x_exact)
    # the same above the floor is a breakdown
    with pytest.raises(O.CGBreakdown):
        cg_residual_form(lambda v: A @ v, b, 6, dot, axpy, perturb=lambda k, den: -1.0 if k == 1 else den)
