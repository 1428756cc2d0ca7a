"""Pins of the oracle's Toeplitz / PSF form of the non-uniform transform pair
(Sec. 2.2 footnote, Fig. 4) and of its exact gridding, against an explicit
brute-force NDFT matrix (CPU only)."""
import numpy as np
import pytest

import oracle as O
import synth as S


def ndft_matrix(kx, ky, N):
    """Dense A: row s, column (y, x): (2N)^-1 exp(-2 pi i (kx x + ky y)), built by loops."""
    A = np.zeros((len(kx), N * N), complex)
    for s in range(len(kx)):
        for y in range(N):
            for x in range(N):
                A[s, y * N + x] = np.exp(-2j * np.pi * (kx[s] * x + ky[s] * y)) / (2 * N)
    return A


def toeplitz(P, x, N, G):
    return O.crop_img(O.ifft2u(P * O.fft2u(O.pad_img(x, G))), N)


def trajectories(N):
    rng = np.random.default_rng(N)
    yield rng.uniform(-0.5, 0.5, 40), rng.uniform(-0.5, 0.5, 40)
    yield S.radial_trajectory(N, 3, 5, 2)


@pytest.mark.parametrize("N,G", [(4, 8), (6, 12), (8, 16), (4, 7), (5, 13), (6, 18), (8, 27)])
def test_psf_toeplitz_equals_AHA(N, G):
    """On the twofold grid and on every grid G = 2 gamma N >= 2N - 1 of
    Eq. (8) (odd sizes included): the same A^H A."""
    for kx, ky in trajectories(N):
        A = ndft_matrix(kx, ky, N)
        P = O.psf_kernel(kx, ky, N, G)
        assert np.max(np.abs(P.imag)) <= 1e-12 * np.max(np.abs(P.real))
        for seed in range(3):
            x = S.random_complex((N, N), seed)
            ref = (A.conj().T @ (A @ x.reshape(-1))).reshape(N, N)
            got = toeplitz(P.real, x, N, G)
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
            # <x, T x> = |A x|^2 >= 0
            q = np.vdot(x, got)
            assert abs(q.imag) < 1e-12 * abs(q)
            assert abs(q.real - np.linalg.norm(A @ x.reshape(-1)) ** 2) < 1e-12 * q.real


@pytest.mark.parametrize("N,G", [(4, 8), (8, 16), (6, 15), (8, 24)])
def test_grid_data_is_adjoint_ndft(N, G):
    kx, ky = S.radial_trajectory(N, 5, 3, 1)
    A = ndft_matrix(kx, ky, N)
    y = S.random_complex((2, len(kx)), 4)
    Y = O.grid_data(kx, ky, y, N, G)
    for j in range(2):
        ref = (A.conj().T @ y[j]).reshape(N, N)
        np.testing.assert_allclose(O.crop_img(O.ifft2u(Y[j]), N), ref, atol=1e-13)
        np.testing.assert_allclose(O.ndft_adjoint(kx, ky, y[j], N, G), ref, atol=1e-13)


def test_cartesian_truncated_psf_acts_as_mask():
    """For samples on the G grid the truncated PSF and the 0/1 mask give the
    same Toeplitz operator on FOV images (Sec. 2.2 footnote)."""
    N, G = 8, 16
    rows = S.cartesian_rows(G, 3, 4)
    fy, fx = np.nonzero(np.broadcast_to(rows[:, None], (G, G)))
    sy = np.where(fy < G // 2, fy, fy - G) / G
    sx = np.where(fx < G // 2, fx, fx - G) / G
    P = O.psf_kernel(sx, sy, N, G).real
    mask = np.zeros((G, G))
    mask[fy, fx] = 1
    for seed in range(3):
        x = S.random_complex((N, N), 30 + seed)
        a = toeplitz(P, x, N, G)
        b = toeplitz(mask, x, N, G)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_synth_cartesian_samples_are_unitary_dft_of_padded_image():
    """The acquisition convention: Cartesian samples equal U pad(rho c_j)."""
    Y, P, rho, c = S.cartesian_frame(8, 2, seed=5, sigma=0.0, every=2, centre=4)
    ref = P[None] * O.fft2u(O.pad_img(rho[None] * c, 16))
    np.testing.assert_allclose(Y, ref, atol=1e-13)
