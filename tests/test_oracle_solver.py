"""Pins of the oracle's CG and IRGNM (Sec. 2.2, Eqs. (2)-(3)) against dense
linear algebra that shares none of its code, plus the temporal schedule
(Sec. 3.3) (CPU only)."""
import numpy as np
import pytest

import oracle as O
import synth as S


def rand_x(g, seed, scale=1.0):
    return O.XVec(S.random_complex((g.N, g.N), seed, scale),
                  S.random_complex((g.J, g.gc, g.gc), seed + 1, scale))


def dense(apply, g):
    n = g.N * g.N + g.J * g.gc * g.gc
    M = np.zeros((n, n), complex)
    for k in range(n):
        e = np.zeros(n, complex)
        e[k] = 1
        M[:, k] = apply(O.XVec.unflat(e, g)).flat()
    return M


def small_problem(seed=0):
    g = O.Geometry(N=4, J=2)           # n_x = 16 + 2*2*2 = 24
    x = rand_x(g, seed)
    x.chat *= 30.0                      # non-trivial coils despite D^-1
    rng = np.random.default_rng(seed)
    P = (rng.uniform(size=(g.G, g.G)) < 0.6).astype(float)
    return g, x, P


def test_cg_iterate_is_krylov_energy_minimiser():
    g, x, P = small_problem(1)
    alpha = 0.05
    A = dense(lambda d: O.normal(x, d, P, alpha, g), g)
    b = rand_x(g, 40)
    bf = b.flat()
    for k in (1, 3, 6):
        xk = O.cg(lambda d: O.normal(x, d, P, alpha, g), b, k).flat()
        # orthonormal Krylov basis by modified Gram-Schmidt (two passes)
        V = []
        v = bf.copy()
        for _ in range(k):
            for _ in range(2):
                for u in V:
                    v = v - np.vdot(u, v) * u
            V.append(v / np.linalg.norm(v))
            v = A @ V[-1]
        V = np.array(V).T
        ref = V @ np.linalg.solve(V.conj().T @ A @ V, V.conj().T @ bf)
        assert np.linalg.norm(xk - ref) <= 1e-9 * np.linalg.norm(ref)


def test_full_length_cg_solves_system():
    g, x, P = small_problem(2)
    alpha = 0.5
    A = dense(lambda d: O.normal(x, d, P, alpha, g), g)
    assert np.allclose(A, A.conj().T, atol=1e-12)
    b = rand_x(g, 41)
    n = A.shape[0]
    xs = O.cg(lambda d: O.normal(x, d, P, alpha, g), b, 3 * n).flat()
    ref = np.linalg.solve(A, b.flat())
    assert np.linalg.norm(xs - ref) <= 1e-9 * np.linalg.norm(ref)


def test_cg_zero_rhs_and_breakdown():
    g, x, P = small_problem(3)
    z = O.XVec.zeros(g)
    out = O.cg(lambda d: O.normal(x, d, P, 0.1, g), z, 10)
    assert np.count_nonzero(out.flat()) == 0
    with pytest.raises(O.CGBreakdown):
        O.cg(lambda d: d.scale(-1.0), rand_x(g, 5), 3)


def test_newton_step_matches_dense_gauss_newton():
    """One IRGNM step with CG run to convergence equals the dense solution of
    (J^H P J + a I) d = J^H (Y - P F^(x)) - a (x - x_ref), with the Jacobian J
    built from F^ alone by exact central differences (F^ is bilinear)."""
    g, x, P = small_problem(4)
    alpha = 0.3
    x_ref = rand_x(g, 50, 0.5)
    Y = P[None] * S.random_complex((g.J, g.G, g.G), 51)
    n = g.N * g.N + g.J * g.gc * g.gc
    xf = x.flat()
    Jm = np.zeros((g.J * g.G * g.G, n), complex)
    h = 0.5
    for k in range(n):
        e = np.zeros(n, complex)
        e[k] = h
        fp = O.F_hat(O.XVec.unflat(xf + e, g), g).reshape(-1)
        fm = O.F_hat(O.XVec.unflat(xf - e, g), g).reshape(-1)
        Jm[:, k] = (fp - fm) / (2 * h)
    Pw = np.repeat(P[None], g.J, 0).reshape(-1)
    F0 = O.F_hat(x, g).reshape(-1)
    Ad = Jm.conj().T @ (Pw[:, None] * Jm) + alpha * np.eye(n)
    bd = Jm.conj().T @ (Y.reshape(-1) - Pw * F0) - alpha * (xf - x_ref.flat())
    ref = np.linalg.solve(Ad, bd)
    b = O.newton_rhs(x, x_ref, Y, P, alpha, g)
    np.testing.assert_allclose(b.flat(), bd, atol=1e-12 * np.linalg.norm(bd))
    d = O.cg(lambda v: O.normal(x, v, P, alpha, g), b, 4 * n).flat()
    assert np.linalg.norm(d - ref) <= 1e-8 * np.linalg.norm(ref)


def test_rhs_vanishes_at_truth_with_noiseless_data():
    """At x^ = x^_true with noiseless data and x^_prev = x^_true the IRGNM
    right-hand side is zero and the step is zero."""
    g = O.Geometry(N=16, J=3)
    xt = rand_x(g, 60)
    xt.chat *= 50
    kx, ky = S.radial_trajectory(g.N, 7, 5, 1)
    ct = O.coils(xt, g)
    y = S.simulate_samples(ct * xt.rho[None], kx, ky, g.G)
    Y = O.grid_data(kx, ky, y, g.N, g.G)
    P = O.psf_kernel(kx, ky, g.N, g.G).real
    b = O.newton_rhs(xt, xt, Y, P, 0.25, g)
    scale = np.linalg.norm(O.DFH(xt, Y, g).flat())
    assert np.linalg.norm(b.flat()) <= 1e-12 * scale
    out = O.nlinv_frame(Y, P, xt, xt, g, O.Params(newton_steps=2, cg_iters=5))
    assert np.linalg.norm((out - xt).flat()) <= 1e-10 * np.linalg.norm(xt.flat())


def test_noiseless_phantom_recovery_cartesian():
    """Qualitative pin: a mildly undersampled noiseless Cartesian phantom is
    recovered up to a global complex scale (rho * |c| against the truth)."""
    N, J = 32, 4
    g = O.Geometry(N=N, J=J)
    Y, P, rho, c = S.cartesian_frame(N, J, seed=3, sigma=0.0, every=2, centre=16)
    x = O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g,
                      O.Params(newton_steps=9, cg_iters=30))
    img = O.image(x, g)
    ref = rho * np.sqrt(np.sum(np.abs(c) ** 2, 0))
    s = np.vdot(img, ref) / np.vdot(img, img)
    err = np.linalg.norm(s * img - ref) / np.linalg.norm(ref)
    assert err < 0.1, err


def test_schedule_source_frames():
    assert [O.source_frame(n, 1, 0) for n in range(5)] == [-1, 0, 1, 2, 3]
    assert [O.source_frame(n, 1, 3) for n in range(6)] == [-1, 0, 1, 2, 3, 4]
    # warm-up 0..2 in order, then groups {3,4,5} -> 2, {6,7,8} -> 5, {9} -> 8
    assert [O.source_frame(n, 3, 2) for n in range(10)] == [-1, 0, 1, 2, 2, 2, 5, 5, 5, 8]
    # every source lies in the window [n - delay, n - 1] of Eq. (10)
    for D in (1, 2, 5, 11):
        for l in (0, 1, 5):
            for n in range(l + 1, 60):
                s = O.source_frame(n, D, l)
                assert n - D <= s <= n - 1


def test_stream_delay_one_is_sequential():
    g = O.Geometry(N=8, J=2)
    prm = O.Params(newton_steps=2, cg_iters=3, damping=0.9)
    frames = []
    for n in range(3):
        Y, P, _, _ = S.cartesian_frame(8, 2, seed=7, sigma=1e-3, frame=n)
        frames.append((Y, P))
    xs = O.nlinv_stream(frames, g, prm, delay=1)
    x = O.XVec.initial(g)
    for n, (Y, P) in enumerate(frames):
        x = O.nlinv_frame(Y, P, x, x.scale(0.9), g, prm)
        np.testing.assert_array_equal(x.flat(), xs[n].flat())


def test_stream_last_step_regulariser_exception():
    """Eq. (10)'s exception: frames after the in-order warm-up start from the
    group's source frame, but their last Newton step is regularised towards
    x^_{n-1}.  With delay 1 this is the sequential stream; otherwise a frame's
    first M-1 steps match the simplified schedule exactly and only the last
    step differs, by a Newton step taken from the same point towards another
    regulariser."""
    g = O.Geometry(N=8, J=2)
    prm = O.Params(newton_steps=3, cg_iters=4, damping=0.9)
    frames = [S.cartesian_frame(8, 2, seed=17, sigma=1e-3, frame=n)[:2] for n in range(6)]
    seq = O.nlinv_stream(frames, g, prm, delay=1)
    ex1 = O.nlinv_stream(frames, g, prm, delay=1, last_from_prev=True)
    for a, b in zip(seq, ex1):
        np.testing.assert_array_equal(a.flat(), b.flat())
    D, WU = 3, 1
    simp = O.nlinv_stream(frames, g, prm, delay=D, warmup=WU)
    ex = O.nlinv_stream(frames, g, prm, delay=D, warmup=WU, last_from_prev=True)
    first = min(n for n in range(6) if O.source_frame(n, D, WU) != n - 1)
    for n in range(first):   # identical up to the first frame the exception touches
        np.testing.assert_array_equal(ex[n].flat(), simp[n].flat())
    assert np.linalg.norm((ex[first] - simp[first]).flat()) > 1e-6 * np.linalg.norm(simp[first].flat())
    for n in range(1, 6):
        s = O.source_frame(n, D, WU)
        xs = ex[s]
        if s == n - 1:        # both regularisers are x^_{n-1}: a plain frame
            ref = O.nlinv_frame(*frames[n], xs, xs.scale(0.9), g, prm)
            np.testing.assert_array_equal(ex[n].flat(), ref.flat())
            continue
        # brute force: M-1 steps towards the source, then one step towards n-1
        y = O.nlinv_frame(*frames[n], xs, xs.scale(0.9), g, O.Params(newton_steps=2, cg_iters=4, damping=0.9))
        alpha = prm.alpha0 * prm.q ** 2
        b = O.newton_rhs(y, ex[n - 1].scale(0.9), frames[n][0], frames[n][1], alpha, g)
        d = O.cg(lambda v: O.normal(y, v, frames[n][1], alpha, g), b, 4)
        np.testing.assert_allclose((y + d).flat(), ex[n].flat(), rtol=0, atol=1e-13)
