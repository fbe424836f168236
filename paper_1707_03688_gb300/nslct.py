"""Thin Python binding of libnslct (include/nslct.h).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels. PyTorch supplies device memory and streams. The functions carry
the C names (``nslct_plan``, ``nslct_forward``, ...); ``Plan`` wraps a plan
handle for convenience. If ``libnslct.so`` has not been built, every call
raises ``NslctUnavailable`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnslct.so")

NSLCT_OK = 0
NSLCT_E_ARG = 1
NSLCT_E_NOT_SYMPLECTIC = 2
NSLCT_E_INFEASIBLE = 3
NSLCT_E_SIZE = 4
NSLCT_E_CUDA = 5
NSLCT_E_NOMEM = 6
NSLCT_E_TIMEOUT = 7
NSLCT_E_UNSUPPORTED = 8

NSLCT_H_HA = 0x0
NSLCT_H_LC = 0x1
NSLCT_H_USER = 0x2
NSLCT_PROJECT_SP4 = 0x10
NSLCT_PREC_FP32 = 0x000
NSLCT_PREC_FP64 = 0x100

# every symbol include/nslct.h declares, in declaration order
EXPORTED = (
    "nslct_plan", "nslct_plan_ex", "nslct_derive", "nslct_plan_params", "nslct_plan_info",
    "nslct_forward", "nslct_inverse", "nslct_forward_pass", "nslct_destroy", "nslct_strerror", "nslct_version",
)


class NslctUnavailable(RuntimeError):
    """libnslct.so is missing or failed to load."""


class NslctError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


_lib = None

_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def load(path: str | None = None):
    """Load libnslct.so (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise NslctUnavailable(f"{path} not found; build it with `python -m paper_1707_03688_gb300.build`")
    try:
        lib = ctypes.CDLL(path)
    except OSError as exc:  # pragma: no cover - depends on the machine
        raise NslctUnavailable(f"cannot load {path}: {exc}") from exc
    sig = {
        "nslct_plan": (ctypes.c_int, [ctypes.POINTER(_VP), _PD, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_uint]),
        "nslct_plan_ex": (ctypes.c_int, [ctypes.POINTER(_VP), _PD, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_uint, _PD]),
        "nslct_derive": (ctypes.c_int, [_PD, ctypes.c_uint, _PD, _PD, _PD, _PD, _PD, _PD, _PD]),
        "nslct_plan_params": (ctypes.c_int, [_VP, ctypes.c_int, _PD, _PD, _PD, _PD]),
        "nslct_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_uint), _PD]),
        "nslct_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
        "nslct_inverse": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
        "nslct_forward_pass": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
        "nslct_destroy": (ctypes.c_int, [_VP]),
        "nslct_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "nslct_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().nslct_strerror(int(code)).decode()
    except NslctUnavailable:
        return f"nslct error {code}"


def _check(code: int, where: str):
    if code != NSLCT_OK:
        raise NslctError(code, where)


def _dbl(arr, n):
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError(f"expected {n} doubles, got {a.size}")
    return a, a.ctypes.data_as(_PD)


def _out(n):
    a = np.zeros(n, dtype=np.float64)
    return a, a.ctypes.data_as(_PD)


# ---------------------------------------------------------------- C-named wrappers


def nslct_derive(abcd, flags: int = 0, h_user=None):
    """Host-only planning: returns dict(abcd, H, Bp, C1, C2, objective)."""
    lib = load()
    m, pm = _dbl(abcd, 16)
    h, ph = (None, None) if h_user is None else _dbl(h_user, 4)
    mu, pmu = _out(16)
    outs = [_out(4) for _ in range(4)]
    obj = ctypes.c_double(0.0)
    _check(lib.nslct_derive(pm, ctypes.c_uint(flags), ph, pmu, *[o[1] for o in outs], ctypes.byref(obj)),
           "nslct_derive")
    names = ("H", "Bp", "C1", "C2")
    res = {k: o[0].reshape(2, 2).copy() for k, o in zip(names, outs)}
    res["abcd"] = mu.reshape(4, 4).copy()
    res["objective"] = obj.value
    return res


def nslct_plan(abcd, nx: int, ny: int, dx: float, dy: float, flags: int = 0, h_user=None) -> int:
    """Create a plan on the current CUDA device; returns the opaque handle (int)."""
    lib = load()
    m, pm = _dbl(abcd, 16)
    handle = _VP(0)
    if h_user is not None or (flags & 0x3) == NSLCT_H_USER:
        h, ph = _dbl(h_user, 4)
        rc = lib.nslct_plan_ex(ctypes.byref(handle), pm, int(nx), int(ny), float(dx), float(dy),
                               ctypes.c_uint(flags | (NSLCT_H_USER if h_user is not None else 0)), ph)
    else:
        rc = lib.nslct_plan(ctypes.byref(handle), pm, int(nx), int(ny), float(dx), float(dy), ctypes.c_uint(flags))
    _check(rc, "nslct_plan")
    return handle.value


def nslct_plan_params(plan: int, field: int = 0):
    lib = load()
    outs = [_out(4) for _ in range(4)]
    _check(lib.nslct_plan_params(_VP(plan), int(field), *[o[1] for o in outs]), "nslct_plan_params")
    return {k: o[0].reshape(2, 2).copy() for k, o in zip(("H", "Bp", "C1", "C2"), outs)}


def nslct_plan_info(plan: int):
    lib = load()
    nx, ny, fl = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_uint(0)
    m, pm = _out(16)
    _check(lib.nslct_plan_info(_VP(plan), ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(fl), pm),
           "nslct_plan_info")
    return {"Nx": nx.value, "Ny": ny.value, "flags": fl.value, "abcd": m.reshape(4, 4).copy()}


def _stream_ptr(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return _VP(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check_field(x, nx, ny, dtype, device, name):
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not x.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if device is not None and x.device.index != device:
        raise ValueError(f"{name} is on cuda:{x.device.index}, the plan on cuda:{device}")
    if x.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {x.dtype}")
    if tuple(x.shape) != (nx, ny):
        raise ValueError(f"{name} must have shape {(nx, ny)}, got {tuple(x.shape)}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def nslct_forward(plan: int, x, out, stream=None):
    """out = L x on `stream` (default: the current torch stream of out's device)."""
    _check(load().nslct_forward(_VP(plan), _VP(x.data_ptr()), _VP(out.data_ptr()), _stream_ptr(stream, out.device)),
           "nslct_forward")
    return out


def nslct_inverse(plan: int, x, out, stream=None):
    _check(load().nslct_inverse(_VP(plan), _VP(x.data_ptr()), _VP(out.data_ptr()), _stream_ptr(stream, out.device)),
           "nslct_inverse")
    return out


def nslct_forward_pass(plan: int, k: int, x, out, stream=None):
    """Enqueue pass k (0..4) of the forward chain (profiling / per-pass tests)."""
    _check(load().nslct_forward_pass(_VP(plan), int(k), _VP(x.data_ptr()), _VP(out.data_ptr()),
                                     _stream_ptr(stream, out.device)), "nslct_forward_pass")
    return out


def nslct_destroy(plan: int):
    _check(load().nslct_destroy(_VP(plan)), "nslct_destroy")


def nslct_version() -> str:
    return load().nslct_version().decode()


# ---------------------------------------------------------------- convenience wrapper


class Plan:
    """One ABCD matrix on one Nx x Ny field, on the current CUDA device.

    ``method``: "ha" (Eq. HA24), "lc" (Eqs. LC08/LC10) or an explicit 2x2 ``h``.
    ``precision``: "fp32" (complex64) or "fp64" (complex128).
    ``dx``/``dy`` default to sqrt(2 pi / N) (the paper's sampling condition).
    """

    def __init__(self, abcd, nx: int, ny: int, dx: float | None = None, dy: float | None = None,
                 method: str = "ha", h=None, project: bool = False, precision: str = "fp32"):
        import torch
        self.nx, self.ny = int(nx), int(ny)
        self.dx = float(dx) if dx is not None else math.sqrt(2 * math.pi / self.nx)
        self.dy = float(dy) if dy is not None else math.sqrt(2 * math.pi / self.ny)
        flags = {"ha": NSLCT_H_HA, "lc": NSLCT_H_LC}[method] if h is None else NSLCT_H_USER
        if project:
            flags |= NSLCT_PROJECT_SP4
        if precision == "fp64":
            flags |= NSLCT_PREC_FP64
            self.dtype = torch.complex128
        elif precision == "fp32":
            self.dtype = torch.complex64
        else:
            raise ValueError("precision must be 'fp32' or 'fp64'")
        self.device = torch.cuda.current_device()
        self.flags = flags
        self.handle = None
        self.handle = nslct_plan(abcd, self.nx, self.ny, self.dx, self.dy, flags, h_user=h)

    def params(self):
        return nslct_plan_params(self.handle)

    def info(self):
        return nslct_plan_info(self.handle)

    def _prep(self, x, out):
        import torch
        _check_field(x, self.nx, self.ny, self.dtype, self.device, "input")
        if out is None:
            out = torch.empty_like(x)
        _check_field(out, self.nx, self.ny, self.dtype, self.device, "output")
        return out

    def forward(self, x, out=None, stream=None):
        out = self._prep(x, out)
        return nslct_forward(self.handle, x, out, stream)

    def inverse(self, x, out=None, stream=None):
        out = self._prep(x, out)
        return nslct_inverse(self.handle, x, out, stream)

    def close(self):
        if self.handle:
            nslct_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
