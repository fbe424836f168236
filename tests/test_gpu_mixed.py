"""Split-precision mode (NSLCT_PREC_SPLIT_F16): 4096-point lines as four-step
DFT-64 stages on the tcgen05 tensor cores (FP16 hi/lo operands, FP32
accumulation in TMEM); the other lengths as FP16 hi/lo DFT-16 products.
Parity bound: relative L2 <= 1e-4 against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_03688_gb300 import build as B
    B.build()
    from paper_1707_03688_gb300 import nslct
    nslct.load()
    return nslct


def _run(plan, g, inverse=False):
    x = torch.from_numpy(np.ascontiguousarray(g)).to(torch.complex64).cuda()
    y = plan.inverse(x) if inverse else plan.forward(x)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


def _oracle(plan, g, inverse=False):
    params = O.decompose(plan.info()["abcd"], plan.params()["H"])
    return (O.inverse if inverse else O.forward)(g, params, plan.dx, plan.dy)


@pytest.mark.parametrize("nx,ny", [(256, 256), (512, 512), (1024, 256), (2048, 512), (96, 4096), (128, 64)])
def test_mixed_matches_oracle(N, nx, ny):
    m = I.random_symplectic_abcd(nx + 5 * ny)
    g = I.blob_field(nx, ny, seed=nx + ny, width_range=(2.0, max(3.0, min(nx, ny) / 8)))
    plan = N.Plan(m, nx, ny, precision="mixed")
    out = _run(plan, g)
    assert O.rel_l2(out, _oracle(plan, g)) < TOL_MIXED
    inv = _run(plan, g, inverse=True)
    assert O.rel_l2(inv, _oracle(plan, g, inverse=True)) < TOL_MIXED
    back = _run(plan, out, inverse=True)
    assert O.rel_l2(back, g) < TOL_MIXED


def test_mixed_4096_full_oracle(N):
    g = I.add_white_noise(I.blob_field(4096, 4096, seed=2), sigma=0.05, seed=102)
    plan = N.Plan(I.random_symplectic_abcd(200), 4096, 4096, precision="mixed")
    out = _run(plan, g)
    err = O.rel_l2(out, _oracle(plan, g))
    assert err < TOL_MIXED
    # and it is a different arithmetic from the FP32 path (not silently the same kernels)
    plan32 = N.Plan(I.random_symplectic_abcd(200), 4096, 4096)
    assert O.rel_l2(out, _run(plan32, g)) > 0.0


def test_mixed_subnormal_and_extreme_inputs(N):
    """Butterflies whose largest component is subnormal (the underflowed tails of
    a narrow blob) or zero, next to large values, stay finite and within the
    bound: the per-butterfly power-of-two scale is clamped to FP32's range."""
    nx = ny = 256
    m = I.random_symplectic_abcd(31)
    plan = N.Plan(m, nx, ny, precision="mixed")
    g = I.blob_field(nx, ny, seed=5, width_range=(1.0, 3.0)).astype(np.complex64)
    g[:8, :] = 0.0
    g[8:16, :] = np.float32(1e-42)          # subnormal FP32
    g[16:24, :] = np.float32(3e-39) * (1 + 1j)
    g[100, 100] = 1e6
    out = _run(plan, g.astype(np.complex128))
    assert np.all(np.isfinite(out))
    assert O.rel_l2(out, _oracle(plan, g.astype(np.complex128))) < TOL_MIXED


@pytest.mark.parametrize("nx,ny,method", [(4096, 768, "ha"), (768, 4096, "ha"), (512, 4096, "lc_y")])
def test_mixed_tcgen05_lines_match_oracle(N, nx, ny, method):
    """The tensor-core kernel's tile schedule: 384 tiles over 152 CTAs (pairs of
    tiles and a lone last tile per CTA) along either axis, and the three-pass
    schedule whose row pass runs three 4096-point transforms; forward, inverse
    and reversibility against the oracle, with no expired wait."""
    m = I.random_symplectic_abcd(nx + 7 * ny)
    g = I.blob_field(nx, ny, seed=nx + 3 * ny, width_range=(2.0, 24.0))
    plan = N.Plan(m, nx, ny, precision="mixed", method=method)
    if method == "lc_y":
        assert plan.passes() == 3
    out = _run(plan, g)
    assert O.rel_l2(out, _oracle(plan, g)) < TOL_MIXED
    inv = _run(plan, g, inverse=True)
    assert O.rel_l2(inv, _oracle(plan, g, inverse=True)) < TOL_MIXED
    assert O.rel_l2(_run(plan, out, inverse=True), g) < TOL_MIXED
    assert N.nslct_status(plan.handle) == N.NSLCT_OK
    plan.close()


def test_mixed_tcgen05_batch_equals_single(N):
    """A same-plan batch runs its 4096-point row passes as one tensor-core
    launch over all fields; each field equals its own transform bit for bit."""
    nx, ny, nb = 256, 4096, 3
    plan = N.Plan(I.random_symplectic_abcd(77), nx, ny, precision="mixed")
    xs = torch.stack([torch.from_numpy(I.blob_field(nx, ny, seed=80 + b)).to(torch.complex64) for b in range(nb)]).cuda()
    ys = torch.empty_like(xs)
    N.nslct_forward_many(plan.handle, xs, ys)
    torch.cuda.synchronize()
    for b in range(nb):
        yb = plan.forward(xs[b].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(yb, ys[b])
    plan.close()
