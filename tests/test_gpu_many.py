"""Same-plan batches (nslct_forward_many / nslct_inverse_many /
nslct_backward_many): one launch per pass over the whole batch for the
line-pair kernel, a launch per field otherwise. Checked field by field against
single-field calls (bit for bit where the same kernel runs) and against the
oracle; the parameter gradients of a batch are the sums of the per-field ones."""
from __future__ import annotations

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


def _batch(nb, nx, ny, dt, seed):
    return torch.from_numpy(np.stack([I.blob_field(nx, ny, seed=seed + k) for k in range(nb)])).to(dt).cuda()


@pytest.mark.parametrize("nx,ny,precision,method", [(256, 512, "fp32", "ha"), (1024, 1024, "fp32", "ha"),
                                                    (512, 512, "fp32", "lc_y"), (96, 128, "fp32", "ha"),
                                                    (64, 64, "fp64", "ha")])
def test_forward_inverse_many_equal_single_calls(N, nx, ny, precision, method):
    m = I.random_symplectic_abcd(300 + nx)
    plan = N.Plan(m, nx, ny, precision=precision, method=method)
    x = _batch(5, nx, ny, plan.dtype, seed=nx)
    y = plan.forward(x)
    z = plan.inverse(y)
    torch.cuda.synchronize()
    for b in range(5):
        yb = plan.forward(x[b].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(y[b], yb), b
    assert float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x)) < (2e-5 if precision == "fp32" else 1e-12)
    if nx * ny <= 256 * 512:
        params = O.decompose(plan.info()["abcd"], plan.params()["H"])
        g = x[3].cpu().numpy().astype(np.complex128)
        ref = O.forward(g, params, plan.dx, plan.dy)
        assert O.rel_l2(y[3].cpu().numpy().astype(np.complex128), ref) < (2e-5 if precision == "fp32" else 1e-12)


def test_strided_batch_and_in_place(N):
    nx = ny = 256
    plan = N.Plan(I.random_symplectic_abcd(5), nx, ny)
    big = _batch(6, nx, ny, torch.complex64, seed=1)
    x = big[::2]                          # stride of two fields
    out = torch.empty(3, nx, ny, dtype=torch.complex64, device="cuda")
    plan.forward(x, out=out)
    ref = torch.stack([plan.forward(x[b].contiguous()) for b in range(3)])
    inplace = x.clone()
    plan.forward(inplace, out=inplace)
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and torch.equal(inplace, ref)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_backward_many_sums_parameter_gradients(N, precision):
    nx = ny = 128 if precision == "fp64" else 256
    m = I.random_symplectic_abcd(9)
    plan = N.Plan(m, nx, ny, precision=precision)
    dt = plan.dtype
    x = _batch(4, nx, ny, dt, seed=20)
    yt = _batch(4, nx, ny, dt, seed=40)
    y = plan.forward(x)
    gy = 2 * (y - yt)
    gx, gth, gch = plan.backward(gy, y, want_theta=True, want_chirp=True)
    torch.cuda.synchronize()
    sth = torch.zeros(10, dtype=torch.float64, device="cuda")
    sch = torch.zeros(12, dtype=torch.float64, device="cuda")
    for b in range(4):
        gxb, gthb, gchb = plan.backward(gy[b].contiguous(), y[b].contiguous(), want_theta=True, want_chirp=True)
        torch.cuda.synchronize()
        assert torch.equal(gx[b], gxb)
        sth += gthb
        sch += gchb
    tol = 1e-9 if precision == "fp64" else 1e-6
    assert float(torch.linalg.vector_norm(gth - sth) / torch.linalg.vector_norm(sth)) < tol
    assert float(torch.linalg.vector_norm(gch - sch) / torch.linalg.vector_norm(sch)) < tol


def test_backward_pass_sequence_equals_backward_many(N):
    """Dual passes 0..4 enqueued one by one give nslct_backward_many's grad_in
    exactly (the same launches); a pass outside 0..4 is refused."""
    nx = ny = 256
    plan = N.Plan(I.random_symplectic_abcd(13), nx, ny)
    x = _batch(3, nx, ny, plan.dtype, seed=90)
    y = plan.forward(x)
    gy = 2 * (y - _batch(3, nx, ny, plan.dtype, seed=95))
    gx = torch.empty_like(gy)
    ws = torch.empty_like(gy)
    N.nslct_backward_many(plan.handle, gy, y, gx, workspace=ws)
    ref = gx.clone()
    gx.zero_()
    for k in range(5):
        N.nslct_backward_pass(plan.handle, k, gy, y, gx, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(gx, ref)
    with pytest.raises(N.NslctError) as exc:
        N.nslct_backward_pass(plan.handle, 5, gy, y, gx, workspace=ws)
    assert exc.value.code == N.NSLCT_E_ARG
    plan.close()


def test_autograd_batch(N):
    from paper_1707_03688_gb300.autograd import nslct_transform
    nx = ny = 64
    m = I.random_symplectic_abcd(11)
    th = torch.tensor(O.theta_from_abcd(m), dtype=torch.float64, requires_grad=True)
    x = _batch(3, nx, ny, torch.complex128, seed=60).requires_grad_(True)
    yt = _batch(3, nx, ny, torch.complex128, seed=80)
    h0 = torch.from_numpy(O.ha_search(m))
    y = nslct_transform(x, th, h0, precision="fp64")
    loss = torch.sum(torch.abs(y - yt) ** 2)
    loss.backward()
    d = I.default_spacing(nx)
    ogth = np.zeros(10)
    for b in range(3):
        _, ogx, gthb, _ = O.loss_and_grad(x[b].detach().cpu().numpy(), yt[b].cpu().numpy(), m, h0.numpy(), d, d)
        ogth += gthb
        assert O.rel_l2(x.grad[b].cpu().numpy(), ogx) < 1e-11
    assert O.rel_l2(th.grad.cpu().numpy(), ogth) < 1e-9


def test_many_rejections(N):
    plan = N.Plan(I.random_symplectic_abcd(1), 64, 64)
    x = torch.zeros(2, 64, 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(N.NslctError) as e:   # overlapping fields
        N.load().nslct_forward_many  # noqa: B018
        N._check(N.load().nslct_forward_many(N._VP(plan.handle), 2, N._VP(x.data_ptr()), 100, N._VP(x.data_ptr()),
                                             100, N._VP(0)), "nslct_forward_many")
    assert e.value.code == N.NSLCT_E_ARG
    padded = N.Plan(I.random_symplectic_abcd(1), 64, 64, pad=(128, 128))
    with pytest.raises(N.NslctError) as e:
        padded.forward(x)
    assert e.value.code == N.NSLCT_E_UNSUPPORTED
