"""CPU-side checks of the C-ABI library: it loads, exports every declared
symbol, and its host-only planning (validation, projection, H choice,
decomposition) agrees with the oracle. No kernel runs here."""
from __future__ import annotations

import os
import re

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I
from paper_1707_03688_gb300 import nslct as N
from tests.golden.loader import paper_matrices

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PM = paper_matrices()


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(N.LIB_PATH):
        from paper_1707_03688_gb300 import build as B
        B.build()
    return N.load()


def _declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nslct\w+)\s*\(", text, flags=re.M)
    return names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert "nslct_forward" in names and "nslct_plan" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(N.EXPORTED) == set(names)
    assert N.nslct_version().startswith("nslct")


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(N, "_lib", None)
    with pytest.raises(N.NslctUnavailable):
        N.load("/nonexistent/libnslct.so")


def test_derive_matches_oracle_decomposition(lib):
    mats = [O.project_sp4(m) for m in PM.values()] + [I.random_symplectic_abcd(s) for s in range(12)]
    for m in mats:
        d = N.nslct_derive(m)
        # the plan's factors multiply back to M (Eq. Bnonsym08), checked by the oracle
        params = O.decompose(m, d["H"])
        np.testing.assert_allclose(O.compose_factors(params), m, atol=1e-11)
        for k in ("Bp", "C1", "C2"):
            np.testing.assert_allclose(d[k], params[k], atol=1e-11 * max(1.0, np.max(np.abs(params[k]))))
        assert d["objective"] == pytest.approx(O.ha_objective(m, d["H"]), rel=1e-12)
        # the plan's H search reaches the oracle's optimum of Eq. HA24
        ho = O.ha_search(m)
        assert d["objective"] <= O.ha_objective(m, ho) * (1 + 1e-6)


def test_derive_lc_closed_form(lib):
    for m in [O.project_sp4(PM["M1"]), O.project_sp4(PM["M2"])] + [I.random_symplectic_abcd(50 + s) for s in range(6)]:
        d = N.nslct_derive(m, flags=N.NSLCT_H_LC)
        hl = O.lc_h(m)
        assert hl is not None
        np.testing.assert_allclose(d["H"], hl, atol=1e-12)
        dy = N.nslct_derive(m, flags=N.NSLCT_H_LC_Y)
        hy = O.lc_h(m, only_y=True)
        if hy is not None:
            np.testing.assert_allclose(dy["H"], hy, atol=1e-12)
            assert dy["H"][0, 0] == 0.0 and dy["H"][0, 1] == 0.0 and dy["H"][1, 0] == 0.0


def test_derive_projection_matches_oracle(lib):
    for name, m in PM.items():
        with pytest.raises(N.NslctError) as exc:
            N.nslct_derive(m)
        assert exc.value.code == N.NSLCT_E_NOT_SYMPLECTIC
        d = N.nslct_derive(m, flags=N.NSLCT_PROJECT_SP4)
        np.testing.assert_allclose(d["abcd"], O.project_sp4(m), atol=1e-12)
        assert O.symplectic_residual(d["abcd"]) < 1e-14 * max(1.0, np.max(np.abs(m))) ** 2


def test_derive_user_h_and_errors(lib):
    m = I.random_symplectic_abcd(3)
    h = O.ha_search(m)
    d = N.nslct_derive(m, flags=N.NSLCT_H_USER, h_user=h)
    np.testing.assert_allclose(d["H"], h, atol=0)
    # an H off the feasible plane leaves B - AH non-symmetric
    with pytest.raises(N.NslctError) as exc:
        N.nslct_derive(m, flags=N.NSLCT_H_USER, h_user=h + np.array([[0.3, 0.0], [0.0, 0.0]]))
    assert exc.value.code == N.NSLCT_E_INFEASIBLE
    with pytest.raises(N.NslctError) as exc:
        N.nslct_derive(np.full(16, np.nan))
    assert exc.value.code == N.NSLCT_E_ARG
    # A = 0 with a non-symmetric B: r = 0 and b12 != b21, no symmetric H exists
    b = np.array([[1.0, 2.0], [0.0, 1.0]])
    bad = np.block([[np.zeros((2, 2)), b], [-np.linalg.inv(b).T, np.zeros((2, 2))]])
    assert O.symplectic_residual(bad) < 1e-14
    with pytest.raises(N.NslctError) as exc:
        N.nslct_derive(bad)
    assert exc.value.code == N.NSLCT_E_INFEASIBLE
    with pytest.raises(ValueError):
        O.ha_search(bad)


def test_degenerate_plane_3d_search(lib):
    # gyrator-type matrices have A = cos(phi) I (r = 0) and symmetric B: every
    # symmetric H is feasible and both searches scan all three entries
    m = I.random_symplectic_abcd(9, middle="gyrator")
    r, rhs = O.feasible_plane(m)
    assert np.linalg.norm(r) < 1e-12 and abs(rhs) < 1e-12
    d = N.nslct_derive(m)
    assert d["objective"] <= O.ha_objective(m, O.ha_search(m)) * (1 + 1e-6)
    np.testing.assert_allclose(O.compose_factors(O.decompose(m, d["H"])), m, atol=1e-11)


def test_plan_rejects_bad_sizes_without_touching_the_gpu(lib):
    m = I.random_symplectic_abcd(1)
    for nx, ny in ((100, 64), (64, 165), (8192, 8), (0, 64), (6, 8)):
        with pytest.raises(N.NslctError) as exc:
            N.nslct_plan(m, nx, ny, 0.3, 0.3)
        assert exc.value.code in (N.NSLCT_E_SIZE, N.NSLCT_E_ARG)
    with pytest.raises(N.NslctError) as exc:
        N.nslct_plan(m, 64, 64, -1.0, 0.3)
    assert exc.value.code == N.NSLCT_E_ARG


def test_derive_type2_is_type1_of_the_inverse(lib):
    """NSLCT_TYPE2 reports the type-1 factors of M^-1 with H = -H1, H1 as good
    as the oracle's type-2 choice; the tr(B) rule picks type 2 exactly for tr B < 0."""
    for s in range(4):
        m = I.random_symplectic_abcd(70 + s)
        d2 = N.nslct_derive(m, flags=N.NSLCT_TYPE2)
        p2 = O.plan_type2(m)
        # both searches minimise the same criterion (near-ties may pick nearby H)
        assert O.ha_objective_type2(m, -d2["H"]) <= O.ha_objective_type2(m, p2["H1"]) * (1 + 1e-6)
        mi = O.symplectic_inverse(m)
        p1 = O.decompose(mi, d2["H"])
        for k in ("Bp", "C1", "C2"):
            np.testing.assert_allclose(d2[k], p1[k], atol=1e-9)
        np.testing.assert_allclose(d2["abcd"], m, atol=0)
        dt = N.nslct_derive(m, flags=N.NSLCT_TYPE_BY_TRACE)
        ref = d2 if O.uses_type2(m) else N.nslct_derive(m)
        np.testing.assert_allclose(dt["H"], ref["H"], atol=0)


def test_entry_points_reject_bad_arguments_without_a_gpu(lib):
    """Argument checks that come before any device work."""
    import ctypes
    vp = ctypes.c_void_p
    m = I.random_symplectic_abcd(2)
    mm, pm = N._dbl(m, 16)
    h = vp(0)
    # zero padding: odd field sizes, fields larger than the grid, H given by the caller
    for args in ((101, 100, 128, 128), (100, 100, 64, 128), (0, 100, 128, 128)):
        assert lib.nslct_plan_padded(ctypes.byref(h), pm, *args, 0.3, 0.3, ctypes.c_uint(0)) == N.NSLCT_E_ARG
    assert lib.nslct_plan_padded(ctypes.byref(h), pm, 100, 100, 128, 128, 0.3, 0.3,
                                 ctypes.c_uint(N.NSLCT_H_USER)) == N.NSLCT_E_ARG
    assert lib.nslct_plan_padded(ctypes.byref(h), pm, 100, 100, 128, 128, 0.3, 0.3,
                                 ctypes.c_uint(N.NSLCT_TYPE2)) == N.NSLCT_E_UNSUPPORTED
    # null plans and empty groups
    assert lib.nslct_forward_many(vp(0), 2, vp(0), 0, vp(0), 0, vp(0)) == N.NSLCT_E_ARG
    assert lib.nslct_backward_many(vp(0), 2, 0, vp(0), vp(0), vp(0), vp(0), vp(0), vp(0), vp(0)) == N.NSLCT_E_ARG
    assert lib.nslct_forward_group(0, None, None, None, vp(0)) == N.NSLCT_E_ARG
    assert lib.nslct_selftest_timeout(vp(0), vp(0), vp(0), vp(0)) == N.NSLCT_E_ARG
    assert lib.nslct_plan_shape(vp(0), None, None, None, None) == N.NSLCT_E_ARG
    assert lib.nslct_plan_passes(vp(0)) == 0
    assert lib.nslct_batch_tune(vp(0), vp(0), 1, None, None) == N.NSLCT_E_ARG
    assert lib.nslct_batch_set_split(vp(0), 4) == N.NSLCT_E_ARG
    assert lib.nslct_batch_threads(vp(0)) == 0
    # single passes: a null plan or batch, a pass outside 0..4
    assert lib.nslct_backward_pass(vp(0), 0, 1, 0, vp(0), vp(0), vp(0), vp(0), vp(0)) == N.NSLCT_E_ARG
    assert lib.nslct_backward_pass(vp(0), 5, 1, 0, vp(0), vp(0), vp(0), vp(0), vp(0)) == N.NSLCT_E_ARG
    assert lib.nslct_batch_forward_pass(vp(0), 0, vp(0)) == N.NSLCT_E_ARG
    assert lib.nslct_batch_set_threads(vp(0), 128) == N.NSLCT_E_ARG
    # batches: an unsupported size is refused before any plan is made
    nx = (ctypes.c_int * 1)(100)
    ny = (ctypes.c_int * 1)(128)
    dd = (ctypes.c_double * 1)(0.3)
    b = vp(0)
    assert lib.nslct_plan_batch(ctypes.byref(b), 1, pm, nx, ny, dd, dd, ctypes.c_uint(0)) == N.NSLCT_E_SIZE
    assert lib.nslct_plan_batch(ctypes.byref(b), 1, pm, ny, ny, dd, dd,
                                ctypes.c_uint(N.NSLCT_TYPE2)) == N.NSLCT_E_UNSUPPORTED
    assert lib.nslct_plan_theta(ctypes.byref(h), (ctypes.c_double * 10)(*([0.1] * 10)), None, 64, 64, 0.3, 0.3,
                                ctypes.c_uint(N.NSLCT_TYPE2)) == N.NSLCT_E_UNSUPPORTED
