"""GPU parity of the three-pass schedule used when H = (0,0;0,h).

With H of Eq. LC10 (or H = 0), chi_H does not depend on k_x, so CC^H is a 1D
convolution along y and shares one row pass with CM^{C2} and the first FFT of
CC^{B'}. These tests check that schedule against the oracle (whose chain runs
the four operators of Eq. HA28 literally, with the plan's H), against the
five-pass schedule on the same plan parameters, and its inverse.
"""
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


def _run(plan, g, inverse=False):
    x = torch.from_numpy(np.ascontiguousarray(g)).to(torch.complex64).cuda()
    y = plan.inverse(x) if inverse else plan.forward(x)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


def _oracle(plan, g, inverse=False):
    params = O.decompose(plan.info()["abcd"], plan.params()["H"])
    return (O.inverse if inverse else O.forward)(g, params, plan.dx, plan.dy)


def _abcd_with_a12(seed):
    for s in range(seed, seed + 50):
        m = I.random_symplectic_abcd(s)
        if abs(m[0, 1]) > 0.05 and O.lc_h(m, only_y=True) is not None:
            return m
    raise AssertionError("no ABCD with a12 != 0")


@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 96), (96, 256), (512, 512), (256, 1024)])
def test_lc_y_forward_inverse_match_oracle(N, nx, ny):
    m = _abcd_with_a12(900 + nx + ny)
    plan = N.Plan(m, nx, ny, method="lc_y")
    assert plan.passes() == 3
    h = plan.params()["H"]
    np.testing.assert_allclose(h, O.lc_h(m, only_y=True), rtol=1e-12, atol=1e-12)
    g = I.blob_field(nx, ny, seed=nx * 7 + ny)
    out = _run(plan, g)
    assert O.rel_l2(out, _oracle(plan, g)) < TOL32
    back = _run(plan, out, inverse=True)
    assert O.rel_l2(back, g) < TOL32
    assert O.rel_l2(_run(plan, g, inverse=True), _oracle(plan, g, inverse=True)) < TOL32


@pytest.mark.parametrize("nx,ny", [(64, 128), (768, 384)])
def test_three_passes_equal_five_passes(N, nx, ny):
    m = _abcd_with_a12(950 + nx)
    short = N.Plan(m, nx, ny, method="lc_y")
    full = N.Plan(m, nx, ny, method="lc_y", full_chain=True)
    assert short.passes() == 3 and full.passes() == 5
    np.testing.assert_array_equal(short.params()["H"], full.params()["H"])
    g = I.blob_field(nx, ny, seed=3)
    a, b = _run(short, g), _run(full, g)
    # both are FP32 evaluations of the same operator: each within 2e-5 of the
    # exact result, so within 4e-5 of each other
    assert O.rel_l2(a, b) < 2 * TOL32
    assert O.rel_l2(a, _oracle(full, g)) < TOL32


def test_h_zero_runs_three_passes(N):
    """H = 0 (the user's choice; feasible when B is symmetric and invertible,
    as for the shear-gyrator-shear generator): CC^0 = -I."""
    nx = ny = 128
    m = I.random_symplectic_abcd(21, middle="gyrator")
    assert abs(m[0, 3] - m[1, 2]) < 1e-12 and abs(np.linalg.det(m[:2, 2:])) > 0.05
    plan = N.Plan(m, nx, ny, h=np.zeros((2, 2)))
    assert plan.passes() == 3
    g = I.blob_field(nx, ny, seed=21)
    out = _run(plan, g)
    assert O.rel_l2(out, _oracle(plan, g)) < TOL32
    assert O.rel_l2(_run(plan, out, inverse=True), g) < TOL32


def test_forward_passes_compose(N):
    nx, ny = 256, 128
    m = _abcd_with_a12(77)
    plan = N.Plan(m, nx, ny, method="lc_y")
    g = torch.from_numpy(I.blob_field(nx, ny, seed=77)).to(torch.complex64).cuda()
    out = torch.empty_like(g)
    for k in range(plan.passes()):
        N.nslct_forward_pass(plan.handle, k, g, out)
    with pytest.raises(N.NslctError):
        N.nslct_forward_pass(plan.handle, 3, g, out)
    ref = plan.forward(g)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_fp64_and_ha_plans_keep_five_passes(N):
    m = _abcd_with_a12(5)
    assert N.Plan(m, 64, 64, method="lc_y", precision="fp64").passes() == 5
    p = N.Plan(m, 64, 64)
    h = p.params()["H"]
    assert p.passes() == (3 if h[0, 0] == 0 and h[0, 1] == 0 and h[1, 0] == 0 else 5)


def test_mixed_precision_three_passes(N):
    nx = ny = 512
    m = _abcd_with_a12(31)
    plan = N.Plan(m, nx, ny, method="lc_y", precision="mixed")
    assert plan.passes() == 3
    g = I.blob_field(nx, ny, seed=31)
    assert O.rel_l2(_run(plan, g), _oracle(plan, g)) < 1e-4
