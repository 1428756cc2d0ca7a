"""GB300 (sm_103a) hot path of NLINV real-time MRI reconstruction.

The compute lives in the C-ABI library ``libnlinv.so`` (include/nlinv.h);
``paper_1701_08361_gb300.nlinv`` is its thin ctypes binding.
"""
from . import nlinv  # noqa: F401
from .nlinv import *  # noqa: F401,F403
