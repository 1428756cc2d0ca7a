"""Thin ctypes binding of the C ABI in include/nlinv.h.

Every function here has the C entry point's name and only marshals
arguments: torch tensors become device pointers, the current torch CUDA
stream becomes the cudaStream_t, return codes become NlinvError.  All
computation runs in libnlinv.so; if the library is missing this module
raises on first use.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("NLINV_LIB") or os.path.join(_HERE, "libnlinv.so")

NLINV_OK = 0
NLINV_EINVAL = -1
NLINV_ECUDA = -2
NLINV_ENOMEM = -3
NLINV_ETIMEOUT = -4
NLINV_ENUMERIC = -5
NLINV_EUNSUPPORTED = -6


class NlinvError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {nlinv_strerror(code)} ({code})"
        if code == NLINV_ECUDA:
            msg += f" [{_lib().nlinv_last_cuda_error().decode()}]"
        super().__init__(msg)


class nlinv_params_t(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("J", ctypes.c_int), ("Gc", ctypes.c_int),
        ("newton_steps", ctypes.c_int), ("cg_iters", ctypes.c_int), ("n_turns", ctypes.c_int),
        ("alpha0", ctypes.c_double), ("q", ctypes.c_double), ("damping", ctypes.c_double),
        ("w_a", ctypes.c_double), ("w_l", ctypes.c_double),
        ("spin_limit", ctypes.c_longlong), ("exec_mode", ctypes.c_int),
        ("max_batch", ctypes.c_int), ("G", ctypes.c_int), ("cluster_cs", ctypes.c_int),
    ]


class nlinv_frame_desc_t(ctypes.Structure):
    _fields_ = [
        ("plan", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("turn", ctypes.c_int),
        ("x_prev", ctypes.c_void_p), ("x_out", ctypes.c_void_p), ("rho_out", ctypes.c_void_p),
        ("img_out", ctypes.c_void_p), ("x_last", ctypes.c_void_p),
    ]


class nlinv_stream_desc_t(ctypes.Structure):
    _fields_ = [
        ("plan", ctypes.c_void_p), ("nframes", ctypes.c_int),
        ("Y", ctypes.POINTER(ctypes.c_void_p)), ("turns", ctypes.POINTER(ctypes.c_int)),
        ("x_out", ctypes.POINTER(ctypes.c_void_p)), ("img_out", ctypes.POINTER(ctypes.c_void_p)),
        ("x_init", ctypes.c_void_p), ("delay", ctypes.c_int), ("warmup", ctypes.c_int),
        ("last_from_prev", ctypes.c_int),
    ]


_L = None
_VP = ctypes.c_void_p
_I = ctypes.c_int

_SIGS = {
    "nlinv_default_params": (_I, [ctypes.POINTER(nlinv_params_t), _I, _I]),
    "nlinv_grid_list": (_I, [_VP, _VP, _I]),
    "nlinv_plan": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(nlinv_params_t), _VP, _VP]),
    "nlinv_plan_destroy": (_I, [_VP]),
    "nlinv_plan_sizes": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_I),
                              ctypes.POINTER(_I)]),
    "nlinv_set_psf": (_I, [_VP, _I, _VP, _VP]),
    "nlinv_plan_path": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "nlinv_psf": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "nlinv_grid": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "nlinv_grid_nufft": (_I, [_VP, _I, _VP, _VP, _I, _VP, _VP]),
    "nlinv_median": (_I, [_VP, _I, ctypes.c_longlong, _VP, _VP]),
    "nlinv_apply_DF": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "nlinv_apply_DFH": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "nlinv_apply_normal": (_I, [_VP, _VP, _VP, _I, ctypes.c_double, _VP, _VP]),
    "nlinv_frame": (_I, [_VP, _VP, _I, _VP, _VP, _VP, _VP, _VP]),
    "nlinv_apply_normal_static": (_I, [_I, _I, _I, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP,
                                       ctypes.c_double, _VP, _VP]),
    "nlinv_batch": (_I, [ctypes.POINTER(nlinv_frame_desc_t), _I, _VP]),
    "nlinv_stream_source": (_I, [_I, _I, _I, ctypes.POINTER(_I)]),
    "nlinv_stream_schedule": (_I, [_I, _I, _I, _I, _VP, _VP, _VP]),
    "nlinv_run_streams": (_I, [ctypes.POINTER(nlinv_stream_desc_t), _I, _VP]),
    "nlinv_wait_flag": (_I, [_VP, _VP, _I, ctypes.c_longlong, _VP]),
    "nlinv_set_alpha0": (_I, [_VP, ctypes.c_double]),
    "nlinv_frame_vjp": (_I, [_VP, _VP, _I, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), _VP, _VP]),
    "nlinv_batch_vjp": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "nlinv_sync": (_I, [_VP, _VP]),
    "nlinv_strerror": (ctypes.c_char_p, [_I]),
    "nlinv_last_cuda_error": (ctypes.c_char_p, []),
}


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _L = lib
    return _L


def library():
    """The loaded ctypes library (loads it on first call)."""
    return _lib()


def _check(rc: int, where: str):
    if rc != NLINV_OK:
        raise NlinvError(rc, where)


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t, dtype=torch.complex64, numel=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


def nlinv_strerror(code: int) -> str:
    return _lib().nlinv_strerror(code).decode()


def nlinv_grid_list():
    """The compiled grids as a list of (G, N) pairs."""
    n = _lib().nlinv_grid_list(None, None, 0)
    G, N = (ctypes.c_int * n)(), (ctypes.c_int * n)()
    _lib().nlinv_grid_list(G, N, n)
    return list(zip(list(G), list(N)))


def nlinv_default_params(N: int, J: int) -> nlinv_params_t:
    p = nlinv_params_t()
    _check(_lib().nlinv_default_params(ctypes.byref(p), N, J), "nlinv_default_params")
    return p


class Plan:
    """Owning handle of an nlinv_plan_t with the plan's sizes."""

    def __init__(self, handle, params: nlinv_params_t):
        self.handle = handle
        self.params = params
        nx, G, Gc = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        _check(_lib().nlinv_plan_sizes(handle, ctypes.byref(nx), ctypes.byref(G),
                                       ctypes.byref(Gc)), "nlinv_plan_sizes")
        self.nx, self.G, self.Gc = nx.value, G.value, Gc.value
        self.N, self.J = params.N, params.J

    def close(self):
        if self.handle:
            _lib().nlinv_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nlinv_plan(params: nlinv_params_t, psf=None, stream=None) -> Plan:
    h = _VP()
    G = params.G or 2 * params.N
    ptr = _ptr(psf, torch.float32, params.n_turns * G * G, "psf") if psf is not None else None
    _check(_lib().nlinv_plan(ctypes.byref(h), ctypes.byref(params), ptr, _stream(stream)),
           "nlinv_plan")
    return Plan(h, params)


def nlinv_plan_destroy(plan: Plan):
    plan.close()


def nlinv_plan_path(plan: Plan):
    """(exec_path, cluster_size): 1 per-phase, 2 grid kernel, 3 cluster kernel."""
    path, cs = ctypes.c_int(), ctypes.c_int()
    _check(_lib().nlinv_plan_path(plan.handle, ctypes.byref(path), ctypes.byref(cs)), "nlinv_plan_path")
    return path.value, cs.value


def nlinv_set_psf(plan: Plan, turn: int, psf, stream=None):
    _check(_lib().nlinv_set_psf(plan.handle, turn, _ptr(psf, torch.float32, plan.G * plan.G, "psf"),
                                _stream(stream)), "nlinv_set_psf")


def nlinv_psf(plan: Plan, turn: int, kxy, P_out=None, stream=None):
    S = kxy.shape[0]
    _check(_lib().nlinv_psf(plan.handle, turn, S, _ptr(kxy, torch.float64, 2 * S, "kxy"),
                            _ptr(P_out, torch.float32, plan.G * plan.G, "P_out"),
                            _stream(stream)), "nlinv_psf")


def nlinv_grid(plan: Plan, kxy, y, Y_out, stream=None):
    S = kxy.shape[0]
    _check(_lib().nlinv_grid(plan.handle, S, _ptr(kxy, torch.float64, 2 * S, "kxy"),
                             _ptr(y, numel=plan.J * S, name="y"),
                             _ptr(Y_out, numel=plan.J * plan.G * plan.G, name="Y_out"),
                             _stream(stream)), "nlinv_grid")


def nlinv_grid_nufft(plan: Plan, kxy, y, W: int, Y_out, stream=None):
    S = kxy.shape[0]
    _check(_lib().nlinv_grid_nufft(plan.handle, S, _ptr(kxy, torch.float64, 2 * S, "kxy"),
                                   _ptr(y, numel=plan.J * S, name="y"), int(W),
                                   _ptr(Y_out, numel=plan.J * plan.G * plan.G, name="Y_out"),
                                   _stream(stream)), "nlinv_grid_nufft")


def nlinv_median(imgs, out, stream=None):
    """Pixel-wise median of |img| over the window `imgs` (list of an odd
    number of complex64 device tensors of equal size) into the float32
    device tensor `out`."""
    n = out.numel()
    T = len(imgs)
    arr = (ctypes.c_void_p * max(1, T))(*[_ptr(t, numel=n, name="img") for t in imgs])
    _check(_lib().nlinv_median(arr, T, n, _ptr(out, torch.float32, n, "out"), _stream(stream)), "nlinv_median")


def nlinv_apply_DF(plan: Plan, xhat, dx, z, stream=None):
    _check(_lib().nlinv_apply_DF(plan.handle, _ptr(xhat, numel=plan.nx, name="xhat"),
                                 _ptr(dx, numel=plan.nx, name="dx"),
                                 _ptr(z, numel=plan.J * plan.G * plan.G, name="z"),
                                 _stream(stream)), "nlinv_apply_DF")


def nlinv_apply_DFH(plan: Plan, xhat, z, dx_out, stream=None):
    _check(_lib().nlinv_apply_DFH(plan.handle, _ptr(xhat, numel=plan.nx, name="xhat"),
                                  _ptr(z, numel=plan.J * plan.G * plan.G, name="z"),
                                  _ptr(dx_out, numel=plan.nx, name="dx_out"),
                                  _stream(stream)), "nlinv_apply_DFH")


def nlinv_apply_normal(plan: Plan, xhat, dx, turn: int, alpha: float, out, stream=None):
    _check(_lib().nlinv_apply_normal(plan.handle, _ptr(xhat, numel=plan.nx, name="xhat"),
                                     _ptr(dx, numel=plan.nx, name="dx"), turn, float(alpha),
                                     _ptr(out, numel=plan.nx, name="out"), _stream(stream)),
           "nlinv_apply_normal")


def nlinv_apply_normal_static(N: int, J: int, Gc: int, w_a: float, w_l: float, xhat, dx, psf,
                              alpha: float, out, stream=None):
    """Plan-free normal operator for callers that cannot allocate device
    memory: all of its intermediates live in the library's fixed 16 MiB
    device array (see include/nlinv.h for the size limit and the rule that
    overlapping calls race)."""
    G = 2 * N
    gc = Gc if Gc else G // 4
    nx = N * N + J * gc * gc
    _check(_lib().nlinv_apply_normal_static(N, J, Gc, float(w_a), float(w_l),
                                            _ptr(xhat, numel=nx, name="xhat"),
                                            _ptr(dx, numel=nx, name="dx"),
                                            _ptr(psf, torch.float32, G * G, "psf"), float(alpha),
                                            _ptr(out, numel=nx, name="out"), _stream(stream)),
           "nlinv_apply_normal_static")


def nlinv_frame(plan: Plan, Y, turn: int, x_prev, x_out, rho_out=None, img_out=None, stream=None):
    NN = plan.N * plan.N
    _check(_lib().nlinv_frame(plan.handle, _ptr(Y, numel=plan.J * plan.G * plan.G, name="Y"), turn,
                              _ptr(x_prev, numel=plan.nx, name="x_prev"),
                              _ptr(x_out, numel=plan.nx, name="x_out"),
                              _ptr(rho_out, numel=NN, name="rho_out"),
                              _ptr(img_out, numel=NN, name="img_out"),
                              _stream(stream)), "nlinv_frame")


def nlinv_batch(frames, stream=None):
    """frames: list of dicts with keys plan, Y, turn, x_prev (tensor or None),
    x_out, and optionally rho_out, img_out, x_last (regulariser of the last
    Newton step: an earlier frame's x_out of the same plan, or any finished
    buffer)."""
    arr = (nlinv_frame_desc_t * len(frames))()
    for i, f in enumerate(frames):
        pl = f["plan"]
        NN = pl.N * pl.N
        arr[i].plan = pl.handle
        arr[i].Y = _ptr(f["Y"], numel=pl.J * pl.G * pl.G, name="Y")
        arr[i].turn = int(f.get("turn", 0))
        arr[i].x_prev = _ptr(f.get("x_prev"), numel=pl.nx, name="x_prev")
        arr[i].x_out = _ptr(f["x_out"], numel=pl.nx, name="x_out")
        arr[i].rho_out = _ptr(f.get("rho_out"), numel=NN, name="rho_out")
        arr[i].img_out = _ptr(f.get("img_out"), numel=NN, name="img_out")
        arr[i].x_last = _ptr(f.get("x_last"), numel=pl.nx, name="x_last")
    _check(_lib().nlinv_batch(arr, len(frames), _stream(stream)), "nlinv_batch")


def nlinv_stream_source(n: int, delay: int, warmup: int) -> int:
    """Source frame of frame n under Eq. (10)'s schedule (-1: initial value)."""
    src = ctypes.c_int()
    _check(_lib().nlinv_stream_source(n, delay, warmup, ctypes.byref(src)), "nlinv_stream_source")
    return src.value


def nlinv_stream_schedule(nframes: int, delay: int, warmup: int, last_from_prev: bool = False):
    """(group, source, last) per frame of one stream, as the library runs it."""
    g, s, l = (ctypes.c_int * max(1, nframes))(), (ctypes.c_int * max(1, nframes))(), (ctypes.c_int * max(1, nframes))()
    rc = _lib().nlinv_stream_schedule(nframes, delay, warmup, 1 if last_from_prev else 0, g, s, l)
    if rc < 0:
        raise NlinvError(rc, "nlinv_stream_schedule")
    return list(g)[:nframes], list(s)[:nframes], list(l)[:nframes]


def nlinv_run_streams(streams, stream=None):
    """streams: list of dicts {plan, Y: list of device tensors, turns: list of
    ints, x: device tensor [nframes, n_x] (or list of [n_x] tensors) for the
    outputs, img: optional [nframes, N*N], x_init: optional [n_x], delay,
    warmup, last_from_prev: optional bool}."""
    keep = []
    arr = (nlinv_stream_desc_t * len(streams))()
    for i, s in enumerate(streams):
        pl = s["plan"]
        nf = len(s["Y"])
        NN = pl.N * pl.N
        Y = (ctypes.c_void_p * nf)(*[_ptr(y, numel=pl.J * pl.G * pl.G, name="Y") for y in s["Y"]])
        T = (ctypes.c_int * nf)(*[int(t) for t in s["turns"]])
        X = (ctypes.c_void_p * nf)(*[_ptr(s["x"][n], numel=pl.nx, name="x") for n in range(nf)])
        keep += [Y, T, X]
        arr[i].plan = pl.handle
        arr[i].nframes = nf
        arr[i].Y = ctypes.cast(Y, ctypes.POINTER(ctypes.c_void_p))
        arr[i].turns = ctypes.cast(T, ctypes.POINTER(ctypes.c_int))
        arr[i].x_out = ctypes.cast(X, ctypes.POINTER(ctypes.c_void_p))
        if s.get("img") is not None:
            I = (ctypes.c_void_p * nf)(*[_ptr(s["img"][n], numel=NN, name="img") for n in range(nf)])
            keep.append(I)
            arr[i].img_out = ctypes.cast(I, ctypes.POINTER(ctypes.c_void_p))
        arr[i].x_init = _ptr(s.get("x_init"), numel=pl.nx, name="x_init")
        arr[i].delay = int(s["delay"])
        arr[i].warmup = int(s["warmup"])
        arr[i].last_from_prev = 1 if s.get("last_from_prev") else 0
    _check(_lib().nlinv_run_streams(arr, len(streams), _stream(stream)), "nlinv_run_streams")


def nlinv_set_alpha0(plan: Plan, alpha0: float):
    _check(_lib().nlinv_set_alpha0(plan.handle, float(alpha0)), "nlinv_set_alpha0")


def nlinv_frame_vjp(plan: Plan, Y, turn: int, x_prev, gbar, Ybar_out, xprev_bar_out=None,
                    stream=None) -> float:
    """dL/dY into Ybar_out (and dL/dx_prev into xprev_bar_out) for
    dL/dx^_M = gbar; returns dL/dalpha_0."""
    a0 = ctypes.c_double(0.0)
    _check(_lib().nlinv_frame_vjp(plan.handle, _ptr(Y, numel=plan.J * plan.G * plan.G, name="Y"), turn,
                                  _ptr(x_prev, numel=plan.nx, name="x_prev"),
                                  _ptr(gbar, numel=plan.nx, name="gbar"),
                                  _ptr(Ybar_out, numel=plan.J * plan.G * plan.G, name="Ybar_out"),
                                  ctypes.byref(a0), _ptr(xprev_bar_out, numel=plan.nx, name="xprev_bar_out"),
                                  _stream(stream)), "nlinv_frame_vjp")
    return a0.value


def nlinv_batch_vjp(plan: Plan, Ys, turns, x_prevs, gbars, Ybars, xprev_bars=None, stream=None):
    """nlinv_frame_vjp of several frames (lists of device tensors; x_prevs or
    xprev_bars may be None or hold None entries); returns the list of
    dL/dalpha_0 per frame."""
    B = len(Ys)
    nk = plan.J * plan.G * plan.G
    VP = ctypes.c_void_p * B
    Y = VP(*[_ptr(y, numel=nk, name="Y") for y in Ys])
    T = (ctypes.c_int * B)(*[int(t) for t in turns])
    XP = VP(*[_ptr(x, numel=plan.nx, name="x_prev") for x in x_prevs]) if x_prevs is not None else None
    GB = VP(*[_ptr(g, numel=plan.nx, name="gbar") for g in gbars])
    YB = VP(*[_ptr(y, numel=nk, name="Ybar") for y in Ybars])
    XB = VP(*[_ptr(x, numel=plan.nx, name="xprev_bar") for x in xprev_bars]) if xprev_bars is not None else None
    a0 = (ctypes.c_double * B)()
    _check(_lib().nlinv_batch_vjp(plan.handle, B, Y, T, XP, GB, YB, a0, XB, _stream(stream)),
           "nlinv_batch_vjp")
    return list(a0)


def nlinv_wait_flag(plan: Plan, flag, expected: int, spin_limit: int, stream=None):
    _check(_lib().nlinv_wait_flag(plan.handle, _ptr(flag, torch.int32, 1, "flag"), expected,
                                  spin_limit, _stream(stream)), "nlinv_wait_flag")


def nlinv_sync(plan: Plan, stream=None) -> int:
    """Synchronise the stream; return the plan's latched device error code
    (0 if none) without raising, so callers can test for it."""
    return _lib().nlinv_sync(plan.handle, _stream(stream))
