"""FP64 CPU oracle of the NLINV hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct NumPy/SciPy complex128 restatement of the
operators and solver of Schaetz, Voit, Frahm & Uecker, "Accelerated Computing
in MRI -- Real-Time Imaging Using Non-Linear Inverse Reconstruction" (2017).
Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm may import this module; the product path never
does, and nothing here is shared with the CUDA path.

Equation numbers follow their order of appearance in the paper:
  Eq. (1)      NLINV objective  ||F x - y||^2 + alpha ||W (x - x_prev)||^2   (Sec. 2.2)
  Eqs. (2)-(3) IRGNM update with the change of variables x^ = W x, F^ = F o W^-1
  Eq. (4)      normal operator DF^H DF : dx -> (sum_j c_j^* t_j, W_b^-H rho^* t_j)
  Eq. (5)      t_j = F_b^H F_b {c_j drho + rho W_b^-1 dc^_j}
  Eq. (10)     temporal decomposition h(n, m)                            (Sec. 3.3)
  Fig. 4       flowchart of the normal operator (W^-1 = iFFT after D_W^-1,
               W^-H = D_W^-1 after FFT; PSF convolution via pad/FFT/P/iFFT/crop)
  Fig. 7       Sobolev weight (1 + 880 |k|^2)^16, -0.5 < k < 0.5
  Sec. 3.2     coil coefficients cropped to G_c = floor(G/4), zero-padded when needed

Conventions (readings of the paper where it is silent; each is listed with
its reason in the design notes):
  * grid G = 2 gamma N of Eq. (8) (G = 2N, gamma = 1, unless chosen); image
    rho on N x N, the FOV sits at rows/cols [0, N) of the G grid (pad writes
    top-left, crop reads top-left);
  * a sample at k (cycles/pixel) is (2N)^-1 sum_r x_r exp(-2 pi i k.r): the
    scale is fixed by the image size, not by the reconstruction grid, so the
    same raw samples can be reconstructed on any G;
  * unitary 2-D DFT U (norm="ortho"), unshifted frequency order;
  * D^-1(f) = (1 + a |2f/G|^2)^(-l/2) with a = 220, l = 32 -- identical to the
    figure's 880 |k|^2 with k = f/G -- applied on the coil grid;
  * coil coefficients c^_j live on a G_c x G_c grid in unshifted order,
    frequency f at index f mod G_c (G_c = G means no crop);
  * x^ = (rho, c^_1..c^_J); inner product Re sum conj(u) v over all parts;
  * alpha_n = alpha_0 q^n; regulariser x_ref = damping * x_prev;
  * sampling enters only as the real PSF multiplier P on the G grid
    (P = mask for Cartesian sampling).
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

_WORKERS = int(os.environ.get("NLINV_ORACLE_THREADS", os.cpu_count() or 1))


def set_workers(n: int) -> None:
    """Thread count for the oracle's library FFTs."""
    global _WORKERS
    _WORKERS = max(1, int(n))


def workers() -> int:
    return _WORKERS


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Geometry:
    """Sizes of one reconstruction: image side N, J channels, coil grid Gc
    (Sec. 3.2: Gc = floor(G/4); Gc = G disables the crop), the Sobolev weight
    constants (Fig. 7) and the grid G = 2 gamma N of Eq. (8) (`grid`; None
    means gamma = 1, G = 2N).  G >= 2N - 1 keeps the PSF convolution of the
    FOV free of wrap-around."""
    N: int
    J: int
    Gc: int | None = None
    w_a: float = 220.0
    w_l: float = 32.0
    grid: int | None = None

    @property
    def G(self) -> int:
        return 2 * self.N if self.grid is None else self.grid

    @property
    def gc(self) -> int:
        return self.G // 4 if self.Gc is None else self.Gc


def freqs(n: int) -> np.ndarray:
    """Signed frequency of each index of an unshifted n-point DFT grid."""
    i = np.arange(n)
    return np.where(i < (n + 1) // 2, i, i - n)


def sobolev_inv_weight(geom: Geometry) -> np.ndarray:
    """Diagonal D_W^-1 on the Gc x Gc coil grid (Fig. 4, Fig. 7):
    (1 + a ((2 fx/G)^2 + (2 fy/G)^2))^(-l/2), f the physical frequency."""
    G, Gc = geom.G, geom.gc
    f = freqs(Gc).astype(np.float64) * 2.0 / G
    k2 = f[:, None] ** 2 + f[None, :] ** 2
    return (1.0 + geom.w_a * k2) ** (-geom.w_l / 2.0)


# ---------------------------------------------------------------------------
# grid helpers: unitary DFT, pad / crop (Fig. 4)
# ---------------------------------------------------------------------------

def fft2u(x: np.ndarray) -> np.ndarray:
    """Unitary 2-D DFT U over the last two axes."""
    return sfft.fft2(x, norm="ortho", workers=_WORKERS)


def ifft2u(x: np.ndarray) -> np.ndarray:
    """U^H = U^-1 over the last two axes."""
    return sfft.ifft2(x, norm="ortho", workers=_WORKERS)


def pad_img(x: np.ndarray, G: int) -> np.ndarray:
    """Zero-pad an N x N image into the top-left of the G x G grid."""
    N = x.shape[-1]
    out = np.zeros(x.shape[:-2] + (G, G), np.complex128)
    out[..., :N, :N] = x
    return out


def crop_img(z: np.ndarray, N: int) -> np.ndarray:
    """Top-left N x N of a G x G grid (the FOV)."""
    return z[..., :N, :N]


def pad_coef(c: np.ndarray, G: int) -> np.ndarray:
    """Place a Gc x Gc unshifted coefficient grid into the G x G grid:
    frequency f goes to index f mod G, everything else is zero (Sec. 3.2)."""
    Gc = c.shape[-1]
    idx = freqs(Gc) % G
    out = np.zeros(c.shape[:-2] + (G, G), np.complex128)
    out[..., idx[:, None], idx[None, :]] = c
    return out


def crop_coef(z: np.ndarray, Gc: int) -> np.ndarray:
    """Keep frequencies of the Gc x Gc coil grid out of a G x G grid."""
    G = z.shape[-1]
    idx = freqs(Gc) % G
    return z[..., idx[:, None], idx[None, :]]


# ---------------------------------------------------------------------------
# the unknown x^ = (rho, c^) and its inner product
# ---------------------------------------------------------------------------

@dataclass
class XVec:
    """x^ = (rho [N,N], chat [J,Gc,Gc]) (Sec. 2.2)."""
    rho: np.ndarray
    chat: np.ndarray

    def __add__(self, o):
        return XVec(self.rho + o.rho, self.chat + o.chat)

    def __sub__(self, o):
        return XVec(self.rho - o.rho, self.chat - o.chat)

    def scale(self, a):
        return XVec(a * self.rho, a * self.chat)

    def copy(self):
        return XVec(self.rho.copy(), self.chat.copy())

    def flat(self) -> np.ndarray:
        return np.concatenate([self.rho.reshape(-1), self.chat.reshape(-1)])

    @staticmethod
    def unflat(v: np.ndarray, geom: Geometry) -> "XVec":
        N, J, Gc = geom.N, geom.J, geom.gc
        return XVec(v[:N * N].reshape(N, N).copy(),
                    v[N * N:].reshape(J, Gc, Gc).copy())

    @staticmethod
    def zeros(geom: Geometry) -> "XVec":
        return XVec(np.zeros((geom.N, geom.N), np.complex128),
                    np.zeros((geom.J, geom.gc, geom.gc), np.complex128))

    @staticmethod
    def initial(geom: Geometry) -> "XVec":
        """First frame: rho set to unity and coils to zero (Sec. 3.3)."""
        x = XVec.zeros(geom)
        x.rho[:] = 1.0
        return x


def dot(u: XVec, v: XVec) -> float:
    """Real inner product Re <u, v> = Re sum conj(u) v over rho and c^."""
    return float(np.real(np.vdot(u.rho, v.rho) + np.vdot(u.chat, v.chat)))


# ---------------------------------------------------------------------------
# operators (Sec. 2.2, Eqs. (2)-(5), Fig. 4)
# ---------------------------------------------------------------------------

def W_inv(chat: np.ndarray, geom: Geometry) -> np.ndarray:
    """W^-1 on the coil part: D_W^-1, zero-pad to G, inverse FFT, restrict
    to the FOV.  [J,Gc,Gc] -> [J,N,N]."""
    z = pad_coef(sobolev_inv_weight(geom) * chat, geom.G)
    return crop_img(ifft2u(z), geom.N)


def W_invH(v: np.ndarray, geom: Geometry) -> np.ndarray:
    """W^-H, the adjoint of W_inv: pad the FOV image, FFT, keep the coil
    grid, D_W^-1.  [J,N,N] -> [J,Gc,Gc]."""
    z = fft2u(pad_img(v, geom.G))
    return sobolev_inv_weight(geom) * crop_coef(z, geom.gc)


def coils(x: XVec, geom: Geometry) -> np.ndarray:
    """Coil sensitivities c_j = W^-1 c^_j of a point x^."""
    return W_inv(x.chat, geom)


def F_hat(x: XVec, geom: Geometry) -> np.ndarray:
    """F^(x^)_j = U pad(rho c_j): predicted (unsampled) k-space on the G grid."""
    return fft2u(pad_img(x.rho[None] * coils(x, geom), geom.G))


def DF(x: XVec, dx: XVec, geom: Geometry) -> np.ndarray:
    """Derivative of F^ at x^ applied to dx: U pad(c_j drho + rho W^-1 dc^_j)."""
    c = coils(x, geom)
    dc = W_inv(dx.chat, geom)
    return fft2u(pad_img(c * dx.rho[None] + x.rho[None] * dc, geom.G))


def DFH(x: XVec, z: np.ndarray, geom: Geometry) -> XVec:
    """Adjoint of DF at x^ (Eq. (4) without the PSF): with t_j = crop U^H z_j,
    returns (sum_j conj(c_j) t_j, W^-H (conj(rho) t_j))."""
    c = coils(x, geom)
    t = crop_img(ifft2u(z), geom.N)
    return XVec(np.sum(np.conj(c) * t, axis=0),
                W_invH(np.conj(x.rho)[None] * t, geom))


def normal(x: XVec, dx: XVec, P: np.ndarray, alpha: float, geom: Geometry) -> XVec:
    """(DF^H P DF + alpha I) dx: the operator of Eq. (4)/(5) with the
    non-uniform transform pair replaced by the PSF multiplier P on the
    twofold-oversampled grid (Sec. 2.2 footnote), plus the Tikhonov term."""
    return DFH(x, P[None] * DF(x, dx, geom), geom) + dx.scale(alpha)


# ---------------------------------------------------------------------------
# conjugate gradients (Sec. 2.2: CG on each Newton step's linear system)
# ---------------------------------------------------------------------------

class CGBreakdown(RuntimeError):
    pass


def cg(apply, b: XVec, iters: int, trace: list | None = None) -> XVec:
    """Fixed-count conjugate gradients from zero: a = |r|^2 / Re<p,Ap>,
    beta = |r_new|^2 / |r|^2.  Stops early only when |r|^2 is exactly 0;
    raises CGBreakdown when Re<p,Ap> <= 0 or is not finite."""
    x = XVec(np.zeros_like(b.rho), np.zeros_like(b.chat))
    r = b.copy()
    p = r.copy()
    rr = dot(r, r)
    for _ in range(iters):
        if rr == 0.0:
            break
        q = apply(p)
        pq = dot(p, q)
        if not (np.isfinite(pq) and pq > 0.0):
            raise CGBreakdown(f"Re<p,Ap> = {pq}")
        a = rr / pq
        x = x + p.scale(a)
        r = r - q.scale(a)
        rr_new = dot(r, r)
        if trace is not None:
            trace.append(dict(rr=rr, pq=pq, a=a, rr_new=rr_new))
        p = r + p.scale(rr_new / rr)
        rr = rr_new
    return x


# ---------------------------------------------------------------------------
# IRGNM frame (Eqs. (2)-(3)) and streams
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Params:
    newton_steps: int = 7
    cg_iters: int = 10
    alpha0: float = 1.0
    q: float = 0.5
    damping: float = 1.0


def newton_rhs(x: XVec, x_ref: XVec, Y: np.ndarray, P: np.ndarray, alpha: float,
               geom: Geometry) -> XVec:
    """Right-hand side of the IRGNM update (Eqs. (2)-(3)):
    DF^H (Y - P F^(x^_n)) - alpha_n (x^_n - x^_ref)."""
    resid = Y - P[None] * F_hat(x, geom)
    return DFH(x, resid, geom) - (x - x_ref).scale(alpha)


def nlinv_frame(Y: np.ndarray, P: np.ndarray, x_init: XVec, x_ref: XVec,
                geom: Geometry, prm: Params = Params(), trace: list | None = None,
                x_ref_last: XVec | None = None) -> XVec:
    """One frame of NLINV: M Newton steps from x^_0 = x_init, each solving
    (DF^H P DF + alpha_n I) delta = rhs by CG and setting x^_{n+1} = x^_n + delta.
    x_ref_last, if given, replaces x_ref in the last Newton step (the
    exception of the temporal decomposition, Sec. 3.3, Eq. (10))."""
    x = x_init.copy()
    M = prm.newton_steps
    for n in range(M):
        alpha = prm.alpha0 * prm.q ** n
        xr = x_ref_last if (x_ref_last is not None and n == M - 1) else x_ref
        b = newton_rhs(x, xr, Y, P, alpha, geom)
        delta = cg(lambda d: normal(x, d, P, alpha, geom), b, prm.cg_iters,
                   trace=None if trace is None else trace)
        x = x + delta
    return x


def image(x: XVec, geom: Geometry) -> np.ndarray:
    """Coil-combined image rho * sqrt(sum_j |c_j|^2)."""
    c = coils(x, geom)
    return x.rho * np.sqrt(np.sum(np.abs(c) ** 2, axis=0))


def source_frame(n: int, delay: int, warmup: int) -> int:
    """Frame whose x^ initialises and regularises frame n under the temporal
    decomposition (Sec. 3.3, Eq. (10)): frames n <= warmup follow strictly in
    order (n - 1); later frames are reconstructed `delay` at a time and each
    uses the most recent frame available when its group starts, i.e. the last
    frame of the previous group (frame `warmup` for the first group), which
    lies within [n - delay, n - 1].  delay = 1 is the sequential stream.
    -1 means the initial value (rho = 1, c = 0)."""
    if n <= warmup:
        return n - 1
    return warmup + ((n - warmup - 1) // delay) * delay


def nlinv_stream(frames, geom: Geometry, prm: Params = Params(),
                 delay: int = 1, warmup: int = 0, last_from_prev: bool = False):
    """Reconstruct a stream of (Y, P) frames in order; frame n starts from
    and is regularised towards damping * x^ of source_frame(n).  With
    last_from_prev, Eq. (10)'s exception holds as well: the last Newton step
    of every frame n > 0 is regularised towards damping * x^_{n-1}, so that
    step of frame n follows the end of frame n - 1."""
    xs = []
    init = XVec.initial(geom)
    for n, (Y, P) in enumerate(frames):
        s = source_frame(n, delay, warmup)
        xp = init if s < 0 else xs[s]
        xl = None
        if last_from_prev and n > 0:
            xl = xs[n - 1].scale(prm.damping)
        xs.append(nlinv_frame(Y, P, xp, xp.scale(prm.damping), geom, prm, x_ref_last=xl))
    return xs


# ---------------------------------------------------------------------------
# non-uniform sampling: exact NDFT, PSF and gridded data (Sec. 2.2 footnote)
# ---------------------------------------------------------------------------

def ndft_adjoint(kx: np.ndarray, ky: np.ndarray, y: np.ndarray, N: int, G: int) -> np.ndarray:
    """A^H y: (A^H y)(r) = (2N)^-1 sum_s y_s exp(+2 pi i k_s . r) on the N x N
    FOV, y [..., S] -> [..., N, N] (the sample scale is fixed by N; G only
    names the reconstruction grid)."""
    r = np.arange(N, dtype=np.float64)
    ex = np.exp(2j * np.pi * np.outer(kx, r))        # [S, x]
    ey = np.exp(2j * np.pi * np.outer(ky, r))        # [S, y]
    return np.einsum("...s,sy,sx->...yx", y, ey, ex, optimize=True) / (2 * N)


def psf_kernel(kx: np.ndarray, ky: np.ndarray, N: int, G: int) -> np.ndarray:
    """PSF P on the G grid for the Toeplitz form of A^H A:
    p(d) = (2N)^-2 sum_s exp(2 pi i k_s . d) for d in [-(N-1), N-1]^2, embedded
    circularly on the G grid (G >= 2N - 1: no offset wraps onto another),
    P = G U p.  Real because p is Hermitian: returned as a complex128 [G, G]
    array whose imaginary part is rounding (callers take .real)."""
    assert G >= 2 * N - 1
    d = np.arange(-(N - 1), N, dtype=np.float64)
    ex = np.exp(2j * np.pi * np.outer(kx, d))        # [S, dx]
    ey = np.exp(2j * np.pi * np.outer(ky, d))        # [S, dy]
    p = (ey.T @ ex) / (4.0 * N * N)                    # [dy, dx]
    emb = np.zeros((G, G), np.complex128)
    idx = d.astype(int) % G
    emb[idx[:, None], idx[None, :]] = p
    P = G * fft2u(emb)
    return P


def grid_data(kx: np.ndarray, ky: np.ndarray, y: np.ndarray, N: int, G: int) -> np.ndarray:
    """Gridded data on the G grid with crop U^H Y_j = A^H y_j exactly:
    Y_j = U pad(A^H y_j)."""
    return fft2u(pad_img(ndft_adjoint(kx, ky, y, N, G), G))


# ---------------------------------------------------------------------------
# gridding by convolution (preprocessing stage, Sec. 3.1): the non-uniform
# adjoint A^H y evaluated with a Kaiser-Bessel kernel on the G grid
# ---------------------------------------------------------------------------

def kb_beta(W: int, sigma: float = 2.0) -> float:
    """Kaiser-Bessel shape for a kernel of W grid points on a grid
    oversampled by sigma (the common choice of the gridding literature:
    beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8))."""
    return float(np.pi * np.sqrt((W / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8))


def kb_kernel(u: np.ndarray, W: int, beta: float) -> np.ndarray:
    """phi(u) = I0(beta sqrt(1 - (2u/W)^2)) for |u| <= W/2 (u in grid points),
    else 0."""
    u = np.asarray(u, dtype=np.float64)
    a = 1.0 - (2.0 * u / W) ** 2
    return np.where(a >= 0.0, np.i0(beta * np.sqrt(np.clip(a, 0.0, None))), 0.0)


def kb_ft(t: np.ndarray, W: int, beta: float) -> np.ndarray:
    """Continuous Fourier transform of kb_kernel, int phi(u) e^{2 pi i u t} du =
    W sinh(s)/s with s = sqrt(beta^2 - (pi W t)^2) (t in cycles per grid
    point, |pi W t| < beta)."""
    s = np.sqrt(beta ** 2 - (np.pi * W * np.asarray(t, dtype=np.float64)) ** 2)
    return W * np.sinh(s) / s


def grid_data_kb(kx: np.ndarray, ky: np.ndarray, y: np.ndarray, N: int, G: int, W: int = 6) -> np.ndarray:
    """Gridded data Y_j = U pad(A^H y_j) with A^H y by convolution gridding.
    The field of view [0, N)^2 has its centre at c = N/2; relative to it the
    image spans at most N/2 <= G/4 in each direction, where the periodic
    copies of the kernel's transform are negligible.
    (1) Each sample y_s is spread onto the W x W grid points f nearest to
        its position p_s = G k_s (periodic on the G grid) with the weight
        phi(u) exp(-2 pi i u.c / G), u = f - p_s (the kernel modulated by the
        centre, so that the transform below is centred on c);
    (2) z(r) = sum_f Z_f e^{2 pi i f.r/G} = G crop_N U^H Z, which equals
        sum_s y_s e^{2 pi i k_s.r} Phi((rx - cx)/G) Phi((ry - cy)/G) up to the
        kernel's aliases, Phi = kb_ft the continuous transform of phi;
    (3) A^H y = z / ((2N) Phi Phi) (deapodisation);
    (4) Y = U pad(A^H y).
    The error against the exact adjoint NDFT falls with the kernel width W."""
    beta = kb_beta(W, G / N)
    J = y.shape[0]
    c = N / 2.0
    Z = np.zeros((J, G, G), np.complex128)
    for s in range(len(kx)):
        px, py = G * kx[s], G * ky[s]
        fx = np.floor(px - W / 2.0).astype(int) + 1 + np.arange(W)   # the W points with |f - p| < W/2
        fy = np.floor(py - W / 2.0).astype(int) + 1 + np.arange(W)
        wx = kb_kernel(fx - px, W, beta) * np.exp(-2j * np.pi * (fx - px) * c / G)
        wy = kb_kernel(fy - py, W, beta) * np.exp(-2j * np.pi * (fy - py) * c / G)
        Z[:, (fy % G)[:, None], (fx % G)[None, :]] += y[:, s, None, None] * (wy[:, None] * wx[None, :])[None]
    z = G * crop_img(ifft2u(Z), N)
    dap = kb_ft((np.arange(N, dtype=np.float64) - c) / G, W, beta)
    img = z / (2 * N * dap[:, None] * dap[None, :])[None]
    return fft2u(pad_img(img, G))


# ---------------------------------------------------------------------------
# post-processing (Sec. 3.1): temporal median filter of the displayed images
# ---------------------------------------------------------------------------

def temporal_median(imgs: np.ndarray) -> np.ndarray:
    """Pixel-wise median over a window of T (odd) consecutive frames of the
    magnitude images |rho ||c|||: imgs [T, ...] complex -> [...] real."""
    imgs = np.asarray(imgs)
    assert imgs.shape[0] % 2 == 1, "odd window"
    return np.median(np.abs(imgs), axis=0)
