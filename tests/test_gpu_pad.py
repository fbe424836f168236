"""GPU parity of zero-padded plans (Secs. 2.A, 5.A): pad-on-load in the first
row pass and crop-on-store in the last, against the oracle's chain on the
zero-padded input, and bit for bit against an unpadded plan on an explicitly
zero-padded field (the same arithmetic after the load)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_03688_gb300 import build as B
    B.build()
    from paper_1707_03688_gb300 import nslct
    nslct.load()
    return nslct


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


# (field, padded grid): pair kernel (power-of-two 256..4096 lines) with even
# and odd row/column offsets, and the general kernel (128, 3 * 2^a)
CASES = [((200, 300), (256, 512)), ((202, 298), (256, 512)), ((100, 100), (128, 192)), ((250, 1000), (384, 1024))]


@pytest.mark.parametrize("shape,grid", CASES)
@pytest.mark.parametrize("method", ["ha", "lc_y"])
def test_padded_forward_inverse_match_oracle(N, shape, grid, method):
    (nx, ny), (px, py) = shape, grid
    m = I.random_symplectic_abcd(nx + py)
    d = float(np.sqrt(2 * np.pi / nx))
    plan = N.Plan(m, nx, ny, dx=d, dy=d, pad=grid, method=method)
    assert plan.in_shape == (nx, ny) and plan.out_shape == (px, py)
    params = O.decompose(plan.info()["abcd"], plan.params()["H"])
    g = I.blob_field(nx, ny, seed=nx + ny)
    out = _host(plan.forward(_dev(g, torch.complex64)))
    ref = O.forward_padded(g, params, d, d, px, py)
    assert O.rel_l2(out, ref) < TOL32
    back = _host(plan.inverse(_dev(out, torch.complex64)))
    assert back.shape == (nx, ny)
    assert O.rel_l2(back, g) < TOL32
    # the same as an unpadded plan on the explicitly zero-padded field
    full = N.Plan(m, px, py, dx=d, dy=d, method=method)
    np.testing.assert_array_equal(full.params()["H"], plan.params()["H"])
    same = _host(full.forward(_dev(O.zero_pad(g, px, py), torch.complex64)))
    assert np.array_equal(out, same)


@pytest.mark.parametrize("shape,grid", [((200, 300), (256, 512)), ((100, 90), (128, 192))])
def test_cropped_output(N, shape, grid):
    (nx, ny), (px, py) = shape, grid
    m = I.random_symplectic_abcd(7 + nx)
    d = float(np.sqrt(2 * np.pi / nx))
    plan = N.Plan(m, nx, ny, dx=d, dy=d, pad=grid, crop=True)
    assert plan.out_shape == (nx, ny)
    params = O.decompose(plan.info()["abcd"], plan.params()["H"])
    g = I.blob_field(nx, ny, seed=3)
    out = _host(plan.forward(_dev(g, torch.complex64)))
    assert O.rel_l2(out, O.forward_padded(g, params, d, d, px, py, crop=True)) < TOL32
    inv = _host(plan.inverse(_dev(out, torch.complex64)))
    assert O.rel_l2(inv, O.inverse_padded(out, params, d, d, px, py, nx, ny)) < TOL32


def test_padded_fp64(N):
    nx, ny, px, py = 50, 60, 64, 96
    m = I.random_symplectic_abcd(12)
    d = float(np.sqrt(2 * np.pi / nx))
    plan = N.Plan(m, nx, ny, dx=d, dy=d, pad=(px, py), precision="fp64")
    params = O.decompose(plan.info()["abcd"], plan.params()["H"])
    g = I.blob_field(nx, ny, seed=12)
    out = _host(plan.forward(_dev(g, torch.complex128)))
    assert O.rel_l2(out, O.forward_padded(g, params, d, d, px, py)) < 1e-12 * (py / 64)
    back = _host(plan.inverse(_dev(out, torch.complex128)))
    assert O.rel_l2(back, g) < 1e-12 * (py / 64)


def test_padded_plan_rejections(N):
    m = I.random_symplectic_abcd(1)
    with pytest.raises(N.NslctError) as e:
        N.Plan(m, 101, 100, pad=(128, 128))          # odd field size
    assert e.value.code == N.NSLCT_E_ARG
    with pytest.raises(N.NslctError) as e:
        N.Plan(m, 200, 100, pad=(128, 128))          # larger than the grid
    assert e.value.code == N.NSLCT_E_ARG
    with pytest.raises(N.NslctError) as e:
        N.Plan(m, 100, 100, pad=(100, 128))          # grid length not supported
    assert e.value.code == N.NSLCT_E_SIZE
    plan = N.Plan(m, 128, 128, pad=(128, 128), crop=True)
    x = torch.zeros(128, 128, dtype=torch.complex64, device="cuda")
    with pytest.raises(N.NslctError) as e:
        N.nslct_forward(plan.handle, x, x)           # in place
    assert e.value.code == N.NSLCT_E_ARG
    with pytest.raises(N.NslctError) as e:
        plan.backward(x, x)
    assert e.value.code == N.NSLCT_E_UNSUPPORTED
