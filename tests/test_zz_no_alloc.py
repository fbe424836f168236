"""nslct_backward_noalloc against nslct_backward.

The no-allocation variant serves callers that cannot allocate device memory
(during CUDA-graph capture, under an allocator that must own every buffer, or
with a fixed budget). It must give the same gradients as nslct_backward, call
after call, while keeping its partial sums in the library's fixed device array
and using the caller's y buffer as its value path. This file is collected
last so that a run stopping at the first failure has run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_03688_gb300 import build as B
    B.build()
    from paper_1707_03688_gb300 import nslct
    nslct.load()
    return nslct


def _rel(a, b):
    a = a.detach().cpu().numpy().astype(np.complex128).ravel()
    b = b.detach().cpu().numpy().astype(np.complex128).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# 4096-point lines fill the library's fixed array (2049 rows per pass, 2048 used)
@pytest.mark.parametrize("nx,ny,precision", [(256, 128, "fp32"), (64, 64, "fp64"), (4096, 64, "fp32"),
                                             (4096, 4096, "fp32")])
def test_noalloc_matches_backward_twice(N, nx, ny, precision):
    lib = N.load()
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    m = I.random_symplectic_abcd(900 + nx)
    h0 = O.ha_search(m)
    plan = N.Plan.from_theta(O.theta_from_abcd(m), nx, ny, h0=h0, precision=precision)
    stream = torch.cuda.current_stream()
    tol = 1e-12 if precision == "fp64" else 2e-5
    for call in range(2):  # two calls in a row share the library's array
        x = torch.from_numpy(I.blob_field(nx, ny, seed=10 * call + 1)).to(dt).cuda()
        yt = torch.from_numpy(I.blob_field(nx, ny, seed=10 * call + 2)).to(dt).cuda()
        y = plan.forward(x)
        gy = 2 * (y - yt)
        # reference: the allocating entry point
        g_ref, th_ref, ch_ref = plan.backward(gy, y, want_theta=True, want_chirp=True)
        # the no-allocation entry point, called through the C ABI
        y_work = y.clone()
        g_new = torch.empty_like(gy)
        th_new = torch.zeros(10, dtype=torch.float64, device="cuda")
        ch_new = torch.zeros(12, dtype=torch.float64, device="cuda")
        rc = lib.nslct_backward_noalloc(ctypes.c_void_p(plan.handle), ctypes.c_void_p(gy.data_ptr()),
                                        ctypes.c_void_p(y_work.data_ptr()), ctypes.c_void_p(g_new.data_ptr()),
                                        ctypes.c_void_p(th_new.data_ptr()), ctypes.c_void_p(ch_new.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))
        assert rc == N.NSLCT_OK, N.strerror(rc)
        torch.cuda.synchronize()
        assert _rel(g_new, g_ref) < tol
        assert _rel(th_new, th_ref) < tol
        assert _rel(ch_new, ch_ref) < tol
        # the value path ran in y_work, which now holds the reconstructed input
        assert _rel(y_work, x) < (1e-11 if precision == "fp64" else 2e-5)
    plan.close()


def test_noalloc_rejects_bad_arguments(N):
    lib = N.load()
    plan = N.Plan(I.random_symplectic_abcd(950), 64, 64)
    g = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
    rc = lib.nslct_backward_noalloc(ctypes.c_void_p(plan.handle), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(0),
                                    ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(0), ctypes.c_void_p(0),
                                    ctypes.c_void_p(0))
    assert rc == N.NSLCT_E_ARG
    # grad_in overlapping y_inout (the value path's buffer) is refused
    y = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
    rc = lib.nslct_backward_noalloc(ctypes.c_void_p(plan.handle), ctypes.c_void_p(g.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(y.data_ptr() + 512),
                                    ctypes.c_void_p(0), ctypes.c_void_p(0), ctypes.c_void_p(0))
    assert rc == N.NSLCT_E_ARG
    plan.close()
