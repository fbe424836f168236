"""GPU parity of the NsLCT-domain filter pipelines of Sec. 5.B: the masked
forward (mask fused into the last pass), Eq. Add04 (two filters, two
inverses) and Eq. Add08 (one inverse of the composed matrix), and the
additivity error of Eq. Add16, against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I
from tests.golden.loader import paper_matrices

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL32 = 2e-5
PM = paper_matrices()


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_03688_gb300 import build as B
    B.build()
    from paper_1707_03688_gb300 import nslct
    nslct.load()
    return nslct


def _dev(a, dt=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def _oparams(plan):
    return O.decompose(plan.info()["abcd"], plan.params()["H"])


@pytest.mark.parametrize("nx,ny,precision,method", [(128, 128, "fp32", "ha"), (512, 256, "fp32", "ha"),
                                                    (256, 256, "fp32", "lc_y"), (96, 64, "fp32", "ha"),
                                                    (64, 64, "fp64", "ha")])
def test_masked_forward(N, nx, ny, precision, method):
    m = I.random_symplectic_abcd(41 + nx)
    plan = N.Plan(m, nx, ny, precision=precision, method=method)
    dt = plan.dtype
    g = I.blob_field(nx, ny, seed=41)
    h = I.gaussian_mask(nx, ny, 0.3, tilt=3.0)
    x, hd = _dev(g, dt), _dev(h, dt)
    y = plan.forward(x)
    ym = plan.forward(x, mask=hd)
    a, b = _host(ym), _host(y * hd)
    tol = 1e-6 if precision == "fp32" else 1e-14
    assert O.rel_l2(a, b) < tol
    ref = h * O.forward(g, _oparams(plan), plan.dx, plan.dy)
    assert O.rel_l2(a, ref) < (TOL32 if precision == "fp32" else 1e-12)


def test_masked_forward_cropped_padded(N):
    nx, ny, px, py = 200, 300, 256, 512
    m = I.random_symplectic_abcd(43)
    d = float(np.sqrt(2 * np.pi / nx))
    plan = N.Plan(m, nx, ny, dx=d, dy=d, pad=(px, py), crop=True)
    g = I.blob_field(nx, ny, seed=43)
    h = I.gaussian_mask(nx, ny, 0.3)
    out = _host(plan.forward(_dev(g), mask=_dev(h)))
    ref = h * O.forward_padded(g, _oparams(plan), d, d, px, py, crop=True)
    assert O.rel_l2(out, ref) < TOL32


def _plans(N, m1, m3, n, d):
    return N.Plan(m1, n, n, dx=d, dy=d), N.Plan(m3, n, n, dx=d, dy=d), N.Plan(m3 @ m1, n, n, dx=d, dy=d)


def test_filter_pipelines_match_oracle(N):
    n, d = 128, 0.22
    m1, m3 = O.project_sp4(PM["M1"]), O.project_sp4(PM["M3"])
    q1, q3, q31 = _plans(N, m1, m3, n, d)
    g = I.hg_field([(1, 2), (3, 1)], n, d)
    h1, h3 = I.gaussian_mask(n, n, 0.3, tilt=2.0), I.gaussian_mask(n, n, 0.4)
    x, h1d, h3d = _dev(g), _dev(h1), _dev(h3)
    y = q3.forward(q1.forward(x, mask=h1d), mask=h3d)
    a04 = _host(q1.inverse(q3.inverse(y)))
    a08 = _host(q31.inverse(y))
    p1, p3, p31 = _oparams(q1), _oparams(q3), _oparams(q31)
    r04 = O.filter_two_domains(g, p1, p3, h1, h3, d, d)
    r08 = O.filter_two_domains_additive(g, p1, p3, p31, h1, h3, d, d)
    assert O.rel_l2(a04, r04) < TOL32
    assert O.rel_l2(a08, r08) < TOL32


def test_additivity_error_matches_oracle(N):
    """NMSE_add (Eq. Add16) of the GPU chains equals the oracle's to 1 %."""
    n, d = 128, 0.22
    m1, m3 = O.project_sp4(PM["M1"]), O.project_sp4(PM["M3"])
    q1, q3, q31 = _plans(N, m1, m3, n, d)
    g = I.hg_field([(1, 2), (3, 1)], n, d)
    x = _dev(g)
    big = _host(q3.forward(q1.forward(x)))
    one = _host(q31.forward(x))
    e_gpu = O.nmse(one, big)
    e_ref = O.nmse_add(g, _oparams(q1), _oparams(q3), _oparams(q31), d, d)
    assert abs(e_gpu - e_ref) < 0.01 * e_ref


def test_masked_forward_rejects_bad_masks(N):
    plan = N.Plan(I.random_symplectic_abcd(5), 64, 64)
    x = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(ValueError):
        plan.forward(x, mask=torch.zeros(64, 32, dtype=torch.complex64, device="cuda"))
    buf = torch.zeros(64 * 64 + 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(N.NslctError) as e:
        N.nslct_forward_masked(plan.handle, x, buf[1:].view(64, 64), out)   # 8-byte aligned only
    assert e.value.code == N.NSLCT_E_ARG
