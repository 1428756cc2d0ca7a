"""Seeded synthetic inputs for NLINV real-time MRI (Schaetz et al. 2017).

This module simulates the *scanner*: an object (moving ellipse phantom), the
receive-coil sensitivities, the sampling pattern (Cartesian rows or the radial
interleaved scheme of Sec. 2.1 / Fig. 3) and the measured k-space samples with
complex Gaussian noise.  It holds none of the reconstruction's arithmetic (no
Sobolev weight, no point-spread function, no gridding, no IRGNM/CG): both the
FP64 oracle and the CUDA path start from what this module returns.

Conventions shared by every consumer (stated, not computed, here):
  * images are arrays indexed [y, x]; pixel r = (x, y) with x, y in [0, N);
  * a k-space position k = (kx, ky) is in cycles/pixel;
  * a sample of coil image m_j at k is  y = G^-1 sum_r m_j(r) exp(-2 pi i k.r),
    the 1/G making Cartesian samples at k = f/G equal the unitary 2-D DFT of
    the zero-padded image on the G x G grid (G = 2N).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "radial_angles", "radial_trajectory", "ellipse_params", "phantom",
    "coil_maps", "simulate_samples", "add_noise", "cartesian_rows",
    "cartesian_frame", "radial_frame", "random_complex",
]


# ---------------------------------------------------------------------------
# sampling patterns
# ---------------------------------------------------------------------------

def radial_angles(K: int, U: int, turn: int) -> np.ndarray:
    """Spoke angles of one frame of the interleaved radial scheme (Sec. 2.1,
    Fig. 3): K spokes spaced 2*pi/K within a frame, successive turns rotated
    by 2*pi/(K*U); turn u = frame index mod U."""
    kappa = np.arange(K, dtype=np.float64)
    return 2.0 * np.pi * kappa / K + 2.0 * np.pi * (turn % U) / (K * U)


def radial_trajectory(N: int, K: int, U: int, turn: int):
    """k-space positions (kx, ky) of one radial frame, N samples per spoke
    (Sec. 4: samples per spoke equal the grid size N), spoke sample m at radius
    (m - N/2)/N cycles/pixel.  Returns two float64 arrays of length K*N,
    spoke-major."""
    theta = radial_angles(K, U, turn)
    rad = (np.arange(N, dtype=np.float64) - N / 2.0) / N
    kx = (np.cos(theta)[:, None] * rad[None, :]).reshape(-1)
    ky = (np.sin(theta)[:, None] * rad[None, :]).reshape(-1)
    return kx, ky


def cartesian_rows(G: int, every: int = 3, centre: int = 16) -> np.ndarray:
    """Boolean [G] of kept phase-encoding rows on the G grid: signed row
    frequency f (unshifted DFT order) kept when f % every == 0 or
    -centre/2 <= f < centre/2."""
    i = np.arange(G)
    f = np.where(i < (G + 1) // 2, i, i - G)
    return (f % every == 0) | ((f >= -(centre // 2)) & (f < centre // 2))


# ---------------------------------------------------------------------------
# object and coils
# ---------------------------------------------------------------------------

def ellipse_params(seed: int, n_ell: int = 10):
    """Random ellipse set (a Shepp-Logan-like layout drawn from `seed`, not
    the canonical table): one body ellipse plus n_ell-1 inner ellipses."""
    rng = np.random.default_rng(seed)
    p = []
    # body: centred, intensity 1
    p.append(dict(cx=0.0, cy=0.0, a=0.42, b=0.36, ang=rng.uniform(0, np.pi),
                  amp=1.0 + 0j, phase0=0.0, move=0.0))
    for _ in range(n_ell - 1):
        amp = rng.uniform(0.2, 1.0) * np.exp(1j * rng.uniform(0.0, 0.3))
        amp *= rng.choice([-0.5, 1.0])
        p.append(dict(cx=rng.uniform(-0.2, 0.2), cy=rng.uniform(-0.2, 0.2),
                      a=rng.uniform(0.05, 0.2), b=rng.uniform(0.05, 0.2),
                      ang=rng.uniform(0, np.pi), amp=amp,
                      phase0=rng.uniform(0, 2 * np.pi), move=0.05))
    return p


def phantom(N: int, seed: int, frame: int = 0, n_ell: int = 10,
            period: float = 50.0) -> np.ndarray:
    """Complex N x N ellipse phantom; inner ellipse centres circle with
    radius 0.05 N and period `period` frames (the moving-phantom stream)."""
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    xs = (x - N / 2.0) / N
    ys = (y - N / 2.0) / N
    img = np.zeros((N, N), np.complex128)
    for e in ellipse_params(seed, n_ell):
        t = 2 * np.pi * frame / period + e["phase0"]
        cx = e["cx"] + e["move"] * np.sin(t)
        cy = e["cy"] + e["move"] * np.cos(t)
        c, s = np.cos(e["ang"]), np.sin(e["ang"])
        u = (xs - cx) * c + (ys - cy) * s
        v = -(xs - cx) * s + (ys - cy) * c
        img += e["amp"] * ((u / e["a"]) ** 2 + (v / e["b"]) ** 2 <= 1.0)
    return img


def coil_maps(N: int, J: int, seed: int, bumps: int = 1) -> np.ndarray:
    """Smooth complex coil sensitivities [J, N, N]: Gaussian bump(s) of width
    0.5 N centred on a circle of radius 0.35 N, times a random phase and a
    slow phase ramp |k_j| <= 0.5/N."""
    rng = np.random.default_rng(seed + 7919)
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    out = np.zeros((J, N, N), np.complex128)
    off = rng.uniform(0, 2 * np.pi)
    for j in range(J):
        for b in range(bumps):
            ang = off + 2 * np.pi * j / J + (rng.uniform(-0.3, 0.3) if b else 0.0)
            rad = 0.35 * N * (1.0 if b == 0 else rng.uniform(0.5, 1.2))
            cx, cy = N / 2 + rad * np.cos(ang), N / 2 + rad * np.sin(ang)
            w = 0.5 * N * (1.0 if b == 0 else rng.uniform(0.4, 0.8))
            g = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * w * w))
            phi = rng.uniform(0, 2 * np.pi)
            kd = rng.uniform(0, 2 * np.pi)
            km = rng.uniform(0, 0.5) / N
            ramp = 2 * np.pi * km * (np.cos(kd) * x + np.sin(kd) * y)
            out[j] += (1.0 if b == 0 else rng.uniform(0.3, 0.8)) * g * np.exp(1j * (phi + ramp))
    return out


# ---------------------------------------------------------------------------
# acquisition
# ---------------------------------------------------------------------------

def simulate_samples(coil_images: np.ndarray, kx: np.ndarray, ky: np.ndarray,
                     G: int) -> np.ndarray:
    """Noise-free samples y[j, s] = G^-1 sum_{y,x} m_j[y,x] exp(-2 pi i (kx x + ky y))
    of coil images m_j [J, N, N] at S positions (FP64, separable sums)."""
    J, N, _ = coil_images.shape
    r = np.arange(N, dtype=np.float64)
    ex = np.exp(-2j * np.pi * np.outer(kx, r))          # [S, N(x)]
    ey = np.exp(-2j * np.pi * np.outer(ky, r))          # [S, N(y)]
    t = coil_images @ ex.T                               # [J, N(y), S]
    return np.einsum("jys,sy->js", t, ey) / G


def add_noise(y: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Complex Gaussian noise with E|n|^2 = sigma^2 (real and imaginary parts
    each N(0, sigma^2/2))."""
    if sigma == 0:
        return y.copy()
    rng = np.random.default_rng(seed + 104729)
    n = rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)
    return y + (sigma / np.sqrt(2.0)) * n


def cartesian_frame(N: int, J: int, seed: int, sigma: float = 1e-3,
                    every: int = 3, centre: int = 16, frame: int = 0):
    """One Cartesian frame on the G = 2N grid: the kept rows' samples placed
    at their grid points.  Returns (Y [J,G,G] complex128, P [G,G] 0/1 mask,
    rho_true, coils_true)."""
    G = 2 * N
    rho = phantom(N, seed, frame)
    c = coil_maps(N, J, seed)
    rows = cartesian_rows(G, every, centre)
    fy_idx, fx_idx = np.nonzero(np.broadcast_to(rows[:, None], (G, G)))
    sy = np.where(fy_idx < G // 2, fy_idx, fy_idx - G) / G
    sx = np.where(fx_idx < G // 2, fx_idx, fx_idx - G) / G
    y = add_noise(simulate_samples(c * rho[None], sx, sy, G), sigma, seed + frame)
    Y = np.zeros((J, G, G), np.complex128)
    Y[:, fy_idx, fx_idx] = y
    P = np.zeros((G, G))
    P[fy_idx, fx_idx] = 1.0
    return Y, P, rho, c


def radial_frame(N: int, J: int, K: int, U: int, frame: int, seed: int,
                 sigma: float = 1e-3, coils: np.ndarray | None = None,
                 bumps: int = 1):
    """Raw samples of one frame of the radial stream: returns
    (kx [S], ky [S], y [J,S] complex128, rho_true, coils_true)."""
    G = 2 * N
    rho = phantom(N, seed, frame)
    c = coil_maps(N, J, seed, bumps) if coils is None else coils
    kx, ky = radial_trajectory(N, K, U, frame % U)
    y = add_noise(simulate_samples(c * rho[None], kx, ky, G), sigma,
                  seed + 31 * frame)
    return kx, ky, y, rho, c


def random_complex(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Complex Gaussian test vector (real/imag each N(0, scale^2/2))."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * (scale / np.sqrt(2.0))
