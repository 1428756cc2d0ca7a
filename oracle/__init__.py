"""FP64 CPU oracle of the NLINV hot path -- test infrastructure only.

Imported only by the tests, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py``.  It shares no code with the CUDA path.
See ``oracle/nlinv.py`` for the operators, solver and their citations.
"""
from .nlinv import *  # noqa: F401,F403
from .nlinv import (Geometry, XVec, Params, CGBreakdown, dot, freqs,  # noqa: F401
                    sobolev_inv_weight, fft2u, ifft2u, pad_img, crop_img,
                    pad_coef, crop_coef, W_inv, W_invH, coils, F_hat, DF, DFH,
                    normal, cg, newton_rhs, nlinv_frame, image, source_frame,
                    nlinv_stream, ndft_adjoint, psf_kernel, grid_data,
                    set_workers, workers)
