"""Oracle work for the full-size parity tests, run in worker processes.

Each job builds one frame's synthetic acquisition (synth), its PSF and
gridded data with the oracle, and the oracle's reconstruction of the frame.
Workers are started with the `spawn` method and import neither torch nor the
CUDA library: this module only calls `synth` and `oracle`.
"""
from __future__ import annotations

import numpy as np

import oracle as O
import synth as S


def init(threads: int) -> None:
    """Worker initialiser: FFT threads of this worker's oracle."""
    O.set_workers(threads)


def radial_inputs(N, J, K, U, n, seed, bumps=1):
    """(Y, P) of frame n of a radial stream: oracle gridding of the synthetic
    samples and the oracle PSF of the frame's trajectory."""
    coils = S.coil_maps(N, J, seed, bumps)
    kx, ky, y, _, _ = S.radial_frame(N, J, K, U, n, seed, 1e-3, coils=coils)
    G = 2 * N
    return O.grid_data(kx, ky, y, N, G), O.psf_kernel(kx, ky, N, G).real


def frame_job(spec):
    """spec: dict(N, J, K, U, n, seed, bumps, x0 (flat complex128 or None)).
    Returns (Y complex64, P float32, x^ of the frame as flat complex128)."""
    N, J = spec["N"], spec["J"]
    g = O.Geometry(N=N, J=J)
    Y, P = radial_inputs(N, J, spec["K"], spec["U"], spec["n"], spec["seed"], spec.get("bumps", 1))
    x0 = O.XVec.initial(g) if spec.get("x0") is None else O.XVec.unflat(spec["x0"], g)
    prm = O.Params()
    x = O.nlinv_frame(Y, P, x0, x0.scale(prm.damping), g, prm)
    return Y.astype(np.complex64), P.astype(np.float32), x.flat()
