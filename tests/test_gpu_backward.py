"""GPU parity of nslct_backward (adjoint + parameter gradients) against the
oracle's gradients (tests/test_oracle_grad.py pins those to finite differences)
and against central finite differences of the GPU's own FP64 forward
(h = 1e-3)."""
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


def _case(nx, ny, seed):
    m = I.random_symplectic_abcd(700 + seed)
    h0 = O.ha_search(m)
    x = I.blob_field(nx, ny, seed=seed, width_range=(1.0, max(2.0, min(nx, ny) / 10)))
    yt = I.blob_field(nx, ny, seed=seed + 1000, width_range=(1.0, max(2.0, min(nx, ny) / 10)))
    return m, h0, x, yt


def _gpu_grads(N, m, h0, x, yt, precision):
    th = O.theta_from_abcd(m)
    plan = N.Plan.from_theta(th, x.shape[0], x.shape[1], h0=h0, precision=precision)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    xd = torch.from_numpy(x).to(dt).cuda()
    y = plan.forward(xd)
    gy = 2 * (y - torch.from_numpy(yt).to(dt).cuda())
    gx, gth, gch = plan.backward(gy, y, want_theta=True, want_chirp=True)
    torch.cuda.synchronize()
    return plan, gx.cpu().numpy().astype(np.complex128), gth.cpu().numpy(), gch.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("nx,ny", [(64, 64), (48, 64)])
def test_fp64_gradients_match_oracle(N, nx, ny):
    m, h0, x, yt = _case(nx, ny, nx + ny)
    plan, gx, gth, gch = _gpu_grads(N, m, h0, x, yt, "fp64")
    _, ogx, ogth, ogch = O.loss_and_grad(x, yt, m, h0, plan.dx, plan.dy)
    assert _rel(gx, ogx) < 1e-11
    assert _rel(gch, ogch) < 1e-9
    assert _rel(gth, ogth) < 1e-9


@pytest.mark.parametrize("nx,ny", [(64, 64), (256, 128), (1024, 1024)])
def test_fp32_gradients_match_oracle(N, nx, ny):
    """The FP32 fields carry a relative rounding error of about eps32 x (log2 N
    radix stages) x (8 FFTs) ~ 6e-8 x 10 x 8 ~ 5e-6, so each chirp gradient (a
    sum of terms w Im(conj(gbar_s) v_s) that cancel by up to 1e6 here) is bounded
    by 2e-5 (4x margin) times the sum of its terms' magnitudes, which the oracle
    computes; the theta gradients inherit the bound through |J|^T."""
    m, h0, x, yt = _case(nx, ny, nx + 2 * ny)
    plan, gx, gth, gch = _gpu_grads(N, m, h0, x, yt, "fp32")
    _, ogx, ogth, ogch = O.loss_and_grad(x, yt, m, h0, plan.dx, plan.dy)
    th = O.theta_from_abcd(m)
    params = O.params_from_theta(th, h0)
    yv = O.forward(x, params, plan.dx, plan.dy)
    _, _, mag = O.chain_vjp(x, 2 * (yv - yt), params, plan.dx, plan.dy, with_abs=True)
    assert _rel(gx, ogx) < 2e-5
    bound_ch = 2e-5 * mag + 1e-6 * np.abs(ogch)
    assert np.all(np.abs(gch - ogch) <= bound_ch), (gch - ogch) / mag
    bound_th = np.abs(O.chirp_jacobian(th, h0)).T @ bound_ch
    assert np.all(np.abs(gth - ogth) <= bound_th)
    # and the bound is meaningful: the vector agrees to about 1e-2 overall (the
    # forward's twiddle powers, up to four roundings deep, enter through y)
    assert _rel(gth, ogth) < 1e-2


def test_grad_in_is_the_inverse_chain(N):
    nx = ny = 256
    m, h0, x, yt = _case(nx, ny, 5)
    plan = N.Plan(m, nx, ny)
    g = torch.from_numpy(yt).to(torch.complex64).cuda()
    y = plan.forward(torch.from_numpy(x).to(torch.complex64).cuda())
    gx, _, _ = plan.backward(g, y, want_theta=False)
    inv = plan.inverse(g)
    torch.cuda.synchronize()
    assert _rel(gx.cpu().numpy(), inv.cpu().numpy()) < 1e-6


def test_theta_gradient_matches_central_differences_fp64(N):
    """Central differences with h = 1e-3 of the GPU FP64 loss, against the GPU
    FP64 adjoint gradient."""
    nx = ny = 64
    m, h0, x, yt = _case(nx, ny, 9)
    plan, _, gth, _ = _gpu_grads(N, m, h0, x, yt, "fp64")
    th = O.theta_from_abcd(m)
    xd = torch.from_numpy(x).cuda()
    ytd = torch.from_numpy(yt).cuda()

    def loss(t):
        p = N.Plan.from_theta(t, nx, ny, h0=h0, precision="fp64")
        v = float(torch.sum(torch.abs(p.forward(xd) - ytd) ** 2).item())
        p.close()
        return v

    def central(h):
        return np.array([(loss(th + h * np.eye(10)[k]) - loss(th - h * np.eye(10)[k])) / (2 * h) for k in range(10)])

    h = 1e-3
    fd = central(h)
    # plain central differences carry an O(h^2) truncation error ...
    assert _rel(gth, fd) < 2e-3
    # ... which Richardson extrapolation with h/2 removes to O(h^4)
    fd_r = (4.0 * central(h / 2) - fd) / 3.0
    assert _rel(gth, fd_r) < 1e-6


def test_autograd_function(N):
    from paper_1707_03688_gb300.autograd import nslct_transform
    nx = ny = 64
    m, h0, x, yt = _case(nx, ny, 11)
    th = torch.tensor(O.theta_from_abcd(m), dtype=torch.float64, requires_grad=True)
    xd = torch.from_numpy(x).to(torch.complex128).cuda().requires_grad_(True)
    y = nslct_transform(xd, th, torch.from_numpy(h0), precision="fp64")
    loss = torch.sum(torch.abs(y - torch.from_numpy(yt).cuda()) ** 2)
    loss.backward()
    _, ogx, ogth, _ = O.loss_and_grad(x, yt, m, h0, I.default_spacing(nx), I.default_spacing(ny))
    assert _rel(xd.grad.cpu().numpy(), ogx) < 1e-11
    assert _rel(th.grad.cpu().numpy(), ogth) < 1e-9


def test_theta_set_equals_a_fresh_theta_plan(N):
    """nslct_plan_theta_set moves a plan to new parameters exactly as
    nslct_plan_theta would plan them (same H rule anchor): the same
    decomposition, the same outputs bit for bit and the same gradients."""
    nx, ny = 128, 96
    m, h0, x, yt = _case(nx, ny, 21)
    th1 = O.theta_from_abcd(m)
    th2 = th1 + np.random.default_rng(5).normal(0.0, 0.05, 10)
    moved = N.Plan.from_theta(th1, nx, ny, h0=h0)
    moved.set_theta(th2)
    fresh = N.Plan.from_theta(th2, nx, ny, h0=h0)
    for k in ("H", "Bp", "C1", "C2"):
        np.testing.assert_array_equal(moved.params()[k], fresh.params()[k])
    np.testing.assert_array_equal(moved.theta(), fresh.theta())
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    ya, yb = moved.forward(xd), fresh.forward(xd)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    gy = 2 * (ya - torch.from_numpy(yt).to(torch.complex64).cuda())
    ga, tha, _ = moved.backward(gy, ya)
    gb, thb, _ = fresh.backward(gy, yb)
    torch.cuda.synchronize()
    assert torch.equal(ga, gb) and torch.equal(tha, thb)
    # a plan without an H anchor cannot be moved; a failed move leaves the plan as it was
    plain = N.Plan(m, nx, ny)
    with pytest.raises(N.NslctError) as exc:
        plain.set_theta(th2)
    assert exc.value.code == N.NSLCT_E_UNSUPPORTED
    bad = th2.copy()
    bad[3:7] = 0.0  # singular L
    with pytest.raises(N.NslctError) as exc:
        moved.set_theta(bad)
    assert exc.value.code == N.NSLCT_E_ARG
    np.testing.assert_array_equal(moved.params()["H"], fresh.params()["H"])
    for p in (moved, fresh, plain):
        p.close()


def test_autograd_reuses_one_plan_across_theta(N):
    """With an anchor h0 the autograd function keeps one plan and moves it to
    each call's theta; two forwards then two backwards (the plan moved between
    a forward and its backward) give the oracle's gradients for each call."""
    from paper_1707_03688_gb300 import autograd as A
    nx = ny = 64
    m, h0, x, yt = _case(nx, ny, 31)
    th0 = O.theta_from_abcd(m)
    ths = [th0, th0 + np.random.default_rng(6).normal(0.0, 0.03, 10)]
    xs, losses = [], []
    for th in ths:
        tht = torch.tensor(th, dtype=torch.float64, requires_grad=True)
        xd = torch.from_numpy(x).to(torch.complex128).cuda().requires_grad_(True)
        y = A.nslct_transform(xd, tht, torch.from_numpy(h0), precision="fp64")
        losses.append(torch.sum(torch.abs(y - torch.from_numpy(yt).cuda()) ** 2))
        xs.append((xd, tht))
    key_h0 = np.ascontiguousarray(h0, dtype=np.float64).reshape(4).tobytes()
    n_cached = sum(1 for k in A._PLANS if k[1:4] == (nx, ny, "fp64") and k[4] == key_h0)
    assert n_cached == 1
    for (xd, tht), loss, th in zip(xs, losses, ths):
        loss.backward()
        _, ogx, ogth, _ = O.loss_and_grad(x, yt, O.abcd_from_theta(th), h0, I.default_spacing(nx),
                                          I.default_spacing(ny))
        assert _rel(xd.grad.cpu().numpy(), ogx) < 1e-11
        assert _rel(tht.grad.cpu().numpy(), ogth) < 1e-9


def test_backward_rejects_misaligned_and_singular_a(N):
    # A = 0 (the 2D DFT): theta is undefined, so only the chirp gradients exist
    z, e = np.zeros((2, 2)), np.eye(2)
    plan = N.Plan(np.block([[z, e], [-e, z]]), 64, 64)
    g = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(N.NslctError) as exc:
        plan.backward(g, g, want_theta=True)
    assert exc.value.code == N.NSLCT_E_UNSUPPORTED
    gx, _, gch = plan.backward(g, g, want_theta=False, want_chirp=True)
    torch.cuda.synchronize()
    assert float(torch.abs(gch).sum()) == 0.0


def test_backward_is_deterministic(N):
    """The CTA partial sums are reduced in a fixed order: repeated calls give
    bit-identical gradients."""
    nx = ny = 256
    m, h0, x, yt = _case(nx, ny, 13)
    plan = N.Plan(m, nx, ny)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    y = plan.forward(xd)
    gy = 2 * (y - torch.from_numpy(yt).to(torch.complex64).cuda())
    first = plan.backward(gy, y, want_theta=True, want_chirp=True)
    for _ in range(3):
        again = plan.backward(gy, y, want_theta=True, want_chirp=True)
        torch.cuda.synchronize()
        for a, b in zip(first, again):
            assert torch.equal(a, b)
