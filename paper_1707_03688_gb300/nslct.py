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
NSLCT_H_LC_Y = 0x3
NSLCT_FULL_CHAIN = 0x20
NSLCT_CROP_OUTPUT = 0x40
NSLCT_TYPE2 = 0x80
NSLCT_TYPE_BY_TRACE = 0x1000
NSLCT_PROJECT_SP4 = 0x10
NSLCT_PREC_FP32 = 0x000
NSLCT_PREC_FP64 = 0x100
NSLCT_PREC_SPLIT_F16 = 0x200

# every symbol include/nslct.h declares, in declaration order
EXPORTED = (
    "nslct_plan", "nslct_plan_ex", "nslct_derive", "nslct_plan_params", "nslct_plan_info",
    "nslct_plan_padded", "nslct_plan_shape",
    "nslct_forward", "nslct_forward_masked", "nslct_forward_group", "nslct_inverse", "nslct_forward_many",
    "nslct_inverse_many",
    "nslct_backward_many", "nslct_backward_pass", "nslct_plan_passes", "nslct_forward_pass", "nslct_backward",
    "nslct_backward_noalloc",
    "nslct_plan_theta", "nslct_plan_theta_set",
    "nslct_plan_theta_get", "nslct_plan_batch", "nslct_batch_size", "nslct_batch_plan", "nslct_batch_bind",
    "nslct_batch_forward", "nslct_batch_capture", "nslct_batch_set_split", "nslct_batch_get_split",
    "nslct_batch_threads", "nslct_batch_set_threads",
    "nslct_batch_tune", "nslct_batch_forward_pass", "nslct_batch_forward_each", "nslct_batch_destroy",
    "nslct_status", "nslct_selftest_timeout", "nslct_destroy", "nslct_strerror", "nslct_version",
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
        "nslct_plan_padded": (ctypes.c_int, [ctypes.POINTER(_VP), _PD, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _D, _D, ctypes.c_uint]),
        "nslct_plan_shape": (ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_int)] * 4),
        "nslct_derive": (ctypes.c_int, [_PD, ctypes.c_uint, _PD, _PD, _PD, _PD, _PD, _PD, _PD]),
        "nslct_plan_params": (ctypes.c_int, [_VP, ctypes.c_int, _PD, _PD, _PD, _PD]),
        "nslct_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_uint), _PD]),
        "nslct_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
        "nslct_inverse": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
        "nslct_plan_passes": (ctypes.c_int, [_VP]),
        "nslct_selftest_timeout": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
        "nslct_forward_masked": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
        "nslct_forward_group": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                               ctypes.POINTER(_VP), _VP]),
        "nslct_forward_many": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_longlong, _VP, ctypes.c_longlong, _VP]),
        "nslct_inverse_many": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_longlong, _VP, ctypes.c_longlong, _VP]),
        "nslct_backward_many": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_longlong, _VP, _VP, _VP, _VP, _VP, _VP,
                                               _VP]),
        "nslct_forward_pass": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
        "nslct_backward_pass": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, _VP, _VP, _VP,
                                               _VP, _VP]),
        "nslct_batch_forward_pass": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
        "nslct_backward": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
        "nslct_backward_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
        "nslct_plan_theta": (ctypes.c_int, [ctypes.POINTER(_VP), _PD, _PD, ctypes.c_int, ctypes.c_int, _D, _D,
                                            ctypes.c_uint]),
        "nslct_plan_theta_get": (ctypes.c_int, [_VP, _PD]),
        "nslct_plan_theta_set": (ctypes.c_int, [_VP, _PD]),
        "nslct_plan_batch": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _PD, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), _PD, _PD, ctypes.c_uint]),
        "nslct_batch_size": (ctypes.c_int, [_VP]),
        "nslct_batch_plan": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
        "nslct_batch_bind": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
        "nslct_batch_forward": (ctypes.c_int, [_VP, _VP]),
        "nslct_batch_capture": (ctypes.c_int, [_VP, _VP]),
        "nslct_batch_forward_each": (ctypes.c_int, [_VP, _VP]),
        "nslct_batch_set_split": (ctypes.c_int, [_VP, ctypes.c_int]),
        "nslct_batch_set_threads": (ctypes.c_int, [_VP, ctypes.c_int]),
        "nslct_batch_get_split": (ctypes.c_int, [_VP]),
        "nslct_batch_threads": (ctypes.c_int, [_VP]),
        "nslct_batch_tune": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_float)]),
        "nslct_batch_destroy": (ctypes.c_int, [_VP]),
        "nslct_status": (ctypes.c_int, [_VP]),
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


def nslct_plan_padded(abcd, nx: int, ny: int, nx_pad: int, ny_pad: int, dx: float, dy: float,
                      flags: int = 0) -> int:
    """Plan on the zero-padded nx_pad x ny_pad grid for an nx x ny input (see include/nslct.h)."""
    lib = load()
    m, pm = _dbl(abcd, 16)
    handle = _VP(0)
    _check(lib.nslct_plan_padded(ctypes.byref(handle), pm, int(nx), int(ny), int(nx_pad), int(ny_pad), float(dx),
                                 float(dy), ctypes.c_uint(flags)), "nslct_plan_padded")
    return handle.value


def nslct_plan_shape(plan: int):
    """((input rows, cols), (output rows, cols)) of a plan."""
    v = [ctypes.c_int(0) for _ in range(4)]
    _check(load().nslct_plan_shape(_VP(plan), *[ctypes.byref(x) for x in v]), "nslct_plan_shape")
    return (v[0].value, v[1].value), (v[2].value, v[3].value)


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


def _check_batch(x, nx, ny, dtype, device, name):
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and x.device.index != device:
        raise ValueError(f"{name} is on cuda:{x.device.index}, the plan on cuda:{device}")
    if x.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {x.dtype}")
    if tuple(x.shape[1:]) != (nx, ny) or x.shape[0] < 1:
        raise ValueError(f"{name} must have shape (B, {nx}, {ny}), got {tuple(x.shape)}")
    if x.stride(2) != 1 or x.stride(1) != ny or (x.shape[0] > 1 and x.stride(0) < nx * ny):
        raise ValueError(f"{name}: each field must be contiguous and fields must not overlap")


def nslct_forward(plan: int, x, out, stream=None):
    """out = L x on `stream` (default: the current torch stream of out's device)."""
    _check(load().nslct_forward(_VP(plan), _VP(x.data_ptr()), _VP(out.data_ptr()), _stream_ptr(stream, out.device)),
           "nslct_forward")
    return out


def nslct_forward_masked(plan: int, x, mask, out, stream=None):
    """out = mask * (L x), the mask multiplied in the last pass."""
    _check(load().nslct_forward_masked(_VP(plan), _VP(x.data_ptr()), _VP(mask.data_ptr()), _VP(out.data_ptr()),
                                       _stream_ptr(stream, out.device)), "nslct_forward_masked")
    return out


def nslct_forward_group(plans, xs, outs, stream=None):
    """out[k] = L_k x[k] for independent transforms, alternated over two streams."""
    n = len(plans)
    ph = (_VP * n)(*[_VP(p) for p in plans])
    pi = (_VP * n)(*[_VP(x.data_ptr()) for x in xs])
    po = (_VP * n)(*[_VP(o.data_ptr()) for o in outs])
    _check(load().nslct_forward_group(n, ph, pi, po, _stream_ptr(stream, outs[0].device)), "nslct_forward_group")
    return outs


def nslct_forward_many(plan: int, x, out, stream=None, inverse: bool = False):
    """The transform (or inverse) of every field of a [B, rows, cols] batch."""
    fn = load().nslct_inverse_many if inverse else load().nslct_forward_many
    _check(fn(_VP(plan), int(x.shape[0]), _VP(x.data_ptr()), int(x.stride(0)), _VP(out.data_ptr()),
              int(out.stride(0)), _stream_ptr(stream, out.device)),
           "nslct_inverse_many" if inverse else "nslct_forward_many")
    return out


def nslct_backward_many(plan: int, grad_out, y, grad_in, grad_theta=None, grad_chirp=None, workspace=None,
                        stream=None):
    """Batched nslct_backward: [B, rows, cols] tensors with one field stride."""
    _check(load().nslct_backward_many(_VP(plan), int(grad_out.shape[0]), int(grad_out.stride(0)), _ptr(grad_out),
                                      _ptr(y), _ptr(grad_in), _ptr(grad_theta), _ptr(grad_chirp), _ptr(workspace),
                                      _stream_ptr(stream, grad_in.device)), "nslct_backward_many")
    return grad_in


def nslct_backward_pass(plan: int, k: int, grad_out, y, grad_in, workspace=None, stream=None):
    """Enqueue dual pass k (0..4) of nslct_backward_many on [B, rows, cols]
    tensors (profiling / per-pass timing; no parameter gradients)."""
    _check(load().nslct_backward_pass(_VP(plan), int(k), int(grad_out.shape[0]), int(grad_out.stride(0)),
                                      _ptr(grad_out), _ptr(y), _ptr(grad_in), _ptr(workspace),
                                      _stream_ptr(stream, grad_in.device)), "nslct_backward_pass")
    return grad_in


def nslct_inverse(plan: int, x, out, stream=None):
    _check(load().nslct_inverse(_VP(plan), _VP(x.data_ptr()), _VP(out.data_ptr()), _stream_ptr(stream, out.device)),
           "nslct_inverse")
    return out


def nslct_forward_pass(plan: int, k: int, x, out, stream=None):
    """Enqueue pass k (0..4) of the forward chain (profiling / per-pass tests)."""
    _check(load().nslct_forward_pass(_VP(plan), int(k), _VP(x.data_ptr()), _VP(out.data_ptr()),
                                     _stream_ptr(stream, out.device)), "nslct_forward_pass")
    return out


def _ptr(t):
    return _VP(t.data_ptr()) if t is not None else _VP(0)


def nslct_backward(plan: int, grad_out, y, grad_in, grad_theta=None, grad_chirp=None, workspace=None, stream=None):
    """grad_in = L^H grad_out; optional device float64 tensors grad_theta (10) and grad_chirp (12)."""
    _check(load().nslct_backward(_VP(plan), _ptr(grad_out), _ptr(y), _ptr(grad_in), _ptr(grad_theta),
                                 _ptr(grad_chirp), _ptr(workspace), _stream_ptr(stream, grad_in.device)),
           "nslct_backward")
    return grad_in


def nslct_backward_noalloc(plan: int, grad_out, y_inout, grad_in, grad_theta=None, grad_chirp=None, stream=None):
    """nslct_backward without any allocation; y_inout is overwritten with L^-1 y (see include/nslct.h)."""
    _check(load().nslct_backward_noalloc(_VP(plan), _ptr(grad_out), _ptr(y_inout), _ptr(grad_in), _ptr(grad_theta),
                                         _ptr(grad_chirp), _stream_ptr(stream, grad_in.device)),
           "nslct_backward_noalloc")
    return grad_in


def nslct_plan_theta(theta, nx: int, ny: int, dx: float, dy: float, h0=None, flags: int = 0) -> int:
    """Plan for M(theta) with H = h0 moved onto the feasible plane (see include/nslct.h)."""
    lib = load()
    t, pt = _dbl(theta, 10)
    h, ph = (None, None) if h0 is None else _dbl(h0, 4)
    handle = _VP(0)
    _check(lib.nslct_plan_theta(ctypes.byref(handle), pt, ph, int(nx), int(ny), float(dx), float(dy),
                                ctypes.c_uint(flags)), "nslct_plan_theta")
    return handle.value


def nslct_plan_theta_set(plan: int, theta):
    """Move a theta plan (made with h0) to new parameters: host FP64 only."""
    _th, pth = _dbl(theta, 10)
    _check(load().nslct_plan_theta_set(_VP(plan), pth), "nslct_plan_theta_set")


def nslct_plan_theta_get(plan: int):
    th, pth = _out(10)
    _check(load().nslct_plan_theta_get(_VP(plan), pth), "nslct_plan_theta_get")
    return th


def nslct_status(plan: int) -> int:
    """NSLCT_OK or NSLCT_E_TIMEOUT (a bounded device wait expired since the last call)."""
    return int(load().nslct_status(_VP(plan)))


def nslct_selftest_timeout(plan: int, x, out, stream=None):
    """Run the first pass with waits that must expire (see include/nslct.h)."""
    _check(load().nslct_selftest_timeout(_VP(plan), _VP(x.data_ptr()), _VP(out.data_ptr()),
                                         _stream_ptr(stream, out.device)), "nslct_selftest_timeout")


def nslct_destroy(plan: int):
    _check(load().nslct_destroy(_VP(plan)), "nslct_destroy")


def nslct_version() -> str:
    return load().nslct_version().decode()


# ---------------------------------------------------------------- convenience wrapper


class Plan:
    """One ABCD matrix on one Nx x Ny field, on the current CUDA device.

    ``method``: "ha" (Eq. HA24), "lc" (Eqs. LC08/LC10) or an explicit 2x2 ``h``.
    ``decomposition``: "type1" (CM-CC-CM-CC, Eq. HA28), "type2" (CC-CM-CC-CM,
    Eq. CCCMCCCM16) or "trace" (the tr(B) rule of Eq. Reversible08).
    ``precision``: "fp32" (complex64) or "fp64" (complex128).
    ``dx``/``dy`` default to sqrt(2 pi / N) (the paper's sampling condition).
    """

    def __init__(self, abcd, nx: int, ny: int, dx: float | None = None, dy: float | None = None,
                 method: str = "ha", h=None, project: bool = False, precision: str = "fp32",
                 full_chain: bool = False, pad=None, crop: bool = False, decomposition: str = "type1"):
        import torch
        self.nx, self.ny = int(nx), int(ny)
        self.dx = float(dx) if dx is not None else math.sqrt(2 * math.pi / self.nx)
        self.dy = float(dy) if dy is not None else math.sqrt(2 * math.pi / self.ny)
        flags = {"ha": NSLCT_H_HA, "lc": NSLCT_H_LC, "lc_y": NSLCT_H_LC_Y}[method] if h is None else NSLCT_H_USER
        if project:
            flags |= NSLCT_PROJECT_SP4
        if full_chain:
            flags |= NSLCT_FULL_CHAIN
        flags |= {"type1": 0, "type2": NSLCT_TYPE2, "trace": NSLCT_TYPE_BY_TRACE}[decomposition]
        if precision == "fp64":
            flags |= NSLCT_PREC_FP64
            self.dtype = torch.complex128
        elif precision == "fp32":
            self.dtype = torch.complex64
        elif precision == "mixed":
            flags |= NSLCT_PREC_SPLIT_F16
            self.dtype = torch.complex64
        else:
            raise ValueError("precision must be 'fp32', 'mixed' or 'fp64'")
        self.device = torch.cuda.current_device()
        self.flags = flags
        self.handle = None
        if pad is None:
            self.handle = nslct_plan(abcd, self.nx, self.ny, self.dx, self.dy, flags, h_user=h)
        else:
            if h is not None:
                raise ValueError("padded plans choose H themselves")
            self.handle = nslct_plan_padded(abcd, self.nx, self.ny, int(pad[0]), int(pad[1]), self.dx, self.dy,
                                            flags | (NSLCT_CROP_OUTPUT if crop else 0))

    @property
    def in_shape(self):
        return nslct_plan_shape(self.handle)[0]

    @property
    def out_shape(self):
        return nslct_plan_shape(self.handle)[1]

    @classmethod
    def from_theta(cls, theta, nx: int, ny: int, h0=None, dx: float | None = None, dy: float | None = None,
                   precision: str = "fp32"):
        """Plan for M(theta) (see nslct_plan_theta)."""
        import torch
        self = cls.__new__(cls)
        self.nx, self.ny = int(nx), int(ny)
        self.dx = float(dx) if dx is not None else math.sqrt(2 * math.pi / self.nx)
        self.dy = float(dy) if dy is not None else math.sqrt(2 * math.pi / self.ny)
        flags = NSLCT_PREC_FP64 if precision == "fp64" else NSLCT_PREC_FP32
        self.dtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.device = torch.cuda.current_device()
        self.flags = flags
        self.handle = None
        self.handle = nslct_plan_theta(theta, self.nx, self.ny, self.dx, self.dy, h0=h0, flags=flags)
        return self

    def theta(self):
        return nslct_plan_theta_get(self.handle)

    def set_theta(self, theta):
        """Move a plan made by from_theta with h0 to new parameters (no allocation, no CUDA call)."""
        nslct_plan_theta_set(self.handle, theta)

    def backward(self, grad_out, y, grad_in=None, want_theta=True, want_chirp=False, workspace=None, stream=None):
        """Returns (grad_in, grad_theta or None, grad_chirp or None); gradients are device float64 tensors.
        3D [B, rows, cols] tensors (one field stride for all) give the batch's
        per-field grad_in and the parameter gradients summed over the batch."""
        import torch
        batched = grad_out.dim() == 3
        chk = (lambda t, name: _check_batch(t, self.nx, self.ny, self.dtype, self.device, name)) if batched else \
            (lambda t, name: _check_field(t, self.nx, self.ny, self.dtype, self.device, name))
        chk(grad_out, "grad_out")
        chk(y, "y")
        if grad_in is None:
            grad_in = torch.empty_like(grad_out)
        chk(grad_in, "grad_in")
        if workspace is not None:
            chk(workspace, "workspace")
        if batched and any(t is not None and (t.shape[0] != grad_out.shape[0] or t.stride(0) != grad_out.stride(0))
                           for t in (y, grad_in, workspace)):
            raise ValueError("batched backward arrays must share batch size and field stride")
        gth = torch.zeros(10, dtype=torch.float64, device=grad_out.device) if want_theta else None
        gch = torch.zeros(12, dtype=torch.float64, device=grad_out.device) if want_chirp else None
        if batched:
            nslct_backward_many(self.handle, grad_out, y, grad_in, gth, gch, workspace, stream)
        else:
            nslct_backward(self.handle, grad_out, y, grad_in, gth, gch, workspace, stream)
        return grad_in, gth, gch

    def passes(self) -> int:
        return int(load().nslct_plan_passes(_VP(self.handle)))

    def params(self):
        return nslct_plan_params(self.handle)

    def info(self):
        return nslct_plan_info(self.handle)

    def _prep(self, x, out, inverse=False):
        import torch
        (ir, ic), (orr, oc) = nslct_plan_shape(self.handle)
        if inverse:
            (ir, ic), (orr, oc) = (orr, oc), (ir, ic)
        if x.dim() == 3:
            # a same-plan batch [B, rows, cols]: fields may be strided along B only
            _check_batch(x, ir, ic, self.dtype, self.device, "input")
            if out is None:
                out = torch.empty((x.shape[0], orr, oc), dtype=x.dtype, device=x.device)
            _check_batch(out, orr, oc, self.dtype, self.device, "output")
            if out.shape[0] != x.shape[0]:
                raise ValueError("input and output batches differ in size")
            return out
        _check_field(x, ir, ic, self.dtype, self.device, "input")
        if out is None:
            out = torch.empty((orr, oc), dtype=x.dtype, device=x.device)
        _check_field(out, orr, oc, self.dtype, self.device, "output")
        return out

    def forward(self, x, out=None, stream=None, mask=None):
        """L x, or mask * (L x) with the mask fused into the last pass. A 3D
        tensor [B, rows, cols] is transformed field by field in batched passes."""
        out = self._prep(x, out)
        if x.dim() == 3:
            if mask is not None:
                raise ValueError("masks apply to single fields")
            return nslct_forward_many(self.handle, x, out, stream)
        if mask is None:
            return nslct_forward(self.handle, x, out, stream)
        _check_field(mask, out.shape[0], out.shape[1], self.dtype, self.device, "mask")
        return nslct_forward_masked(self.handle, x, mask, out, stream)

    def inverse(self, x, out=None, stream=None):
        out = self._prep(x, out, inverse=True)
        if x.dim() == 3:
            return nslct_forward_many(self.handle, x, out, stream, inverse=True)
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


# ---------------------------------------------------------------- batches


def nslct_plan_batch(abcds, nx, ny, dx, dy, flags: int = 0) -> int:
    lib = load()
    n = len(nx)
    m, pm = _dbl(np.asarray(abcds, dtype=np.float64).reshape(n, 16), 16 * n)
    ax = (ctypes.c_int * n)(*[int(v) for v in nx])
    ay = (ctypes.c_int * n)(*[int(v) for v in ny])
    ddx, pdx = _dbl(dx, n)
    ddy, pdy = _dbl(dy, n)
    handle = _VP(0)
    _check(lib.nslct_plan_batch(ctypes.byref(handle), n, pm, ax, ay, pdx, pdy, ctypes.c_uint(flags)),
           "nslct_plan_batch")
    return handle.value


class Batch:
    """Fields of uneven sizes, each with its own ABCD matrix (FP32)."""

    def __init__(self, abcds, shapes, method_flags: int = 0):
        self.shapes = [(int(a), int(b)) for a, b in shapes]
        nx = [a for a, _ in self.shapes]
        ny = [b for _, b in self.shapes]
        dx = [math.sqrt(2 * math.pi / a) for a in nx]
        dy = [math.sqrt(2 * math.pi / b) for b in ny]
        self.dx, self.dy = dx, dy
        self.handle = None
        self.handle = nslct_plan_batch(abcds, nx, ny, dx, dy, method_flags)
        self._bound = None

    def plan_handle(self, i: int) -> int:
        h = _VP(0)
        _check(load().nslct_batch_plan(_VP(self.handle), int(i), ctypes.byref(h)), "nslct_batch_plan")
        return h.value

    def params(self, i: int):
        return nslct_plan_params(self.plan_handle(i))

    def info(self, i: int):
        return nslct_plan_info(self.plan_handle(i))

    def bind(self, ins, outs):
        import torch
        n = len(self.shapes)
        for (nx, ny), a, b in zip(self.shapes, ins, outs):
            _check_field(a, nx, ny, torch.complex64, None, "input")
            _check_field(b, nx, ny, torch.complex64, None, "output")
        pin = (_VP * n)(*[t.data_ptr() for t in ins])
        pout = (_VP * n)(*[t.data_ptr() for t in outs])
        _check(load().nslct_batch_bind(_VP(self.handle), pin, pout), "nslct_batch_bind")
        self._bound = (list(ins), list(outs))

    def capture(self, stream):
        _check(load().nslct_batch_capture(_VP(self.handle), _stream_ptr(stream, None)), "nslct_batch_capture")

    def forward(self, stream=None):
        import torch
        _check(load().nslct_batch_forward(_VP(self.handle), _stream_ptr(stream, torch.cuda.current_device())),
               "nslct_batch_forward")

    def set_split(self, split: int):
        """Fields with min(Nx, Ny) >= split run through their own fused passes."""
        _check(load().nslct_batch_set_split(_VP(self.handle), int(split)), "nslct_batch_set_split")

    def set_threads(self, threads: int):
        """Pin the batched kernels' CTA size (128, 256 or 512)."""
        _check(load().nslct_batch_set_threads(_VP(self.handle), int(threads)), "nslct_batch_set_threads")

    @property
    def split(self) -> int:
        return int(load().nslct_batch_get_split(_VP(self.handle)))

    @property
    def threads(self) -> int:
        """CTA size of the batched kernels (128, 256 or 512)."""
        return int(load().nslct_batch_threads(_VP(self.handle)))

    def tune(self, stream=None, iters: int = 3):
        """Autotune the split on the bound buffers; returns (split, ms per forward)."""
        import torch
        chosen, ms = ctypes.c_int(0), ctypes.c_float(0.0)
        _check(load().nslct_batch_tune(_VP(self.handle), _stream_ptr(stream, torch.cuda.current_device()),
                                       int(iters), ctypes.byref(chosen), ctypes.byref(ms)), "nslct_batch_tune")
        return chosen.value, ms.value

    def forward_pass(self, k: int, stream=None):
        """Enqueue pass k (0..4) of the batch's forward (profiling / per-pass timing)."""
        import torch
        _check(load().nslct_batch_forward_pass(_VP(self.handle), int(k),
                                               _stream_ptr(stream, torch.cuda.current_device())),
               "nslct_batch_forward_pass")

    def forward_each(self, stream=None):
        import torch
        _check(load().nslct_batch_forward_each(_VP(self.handle), _stream_ptr(stream, torch.cuda.current_device())),
               "nslct_batch_forward_each")

    def close(self):
        if self.handle:
            load().nslct_batch_destroy(_VP(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
