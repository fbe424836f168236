"""Pins for the FP64 oracle: checks against what the paper and the mathematics
fix, never against the oracle's own formulas retyped.

* closed forms: the chain for (0,I;-I,0) is the 2D DFT of Eq. BasicDFT16
  (library FFT), for (I,B;0,I) a chirp convolution (library FFT), for (I,0;C,I)
  a chirp multiplication, for I the identity;
* separability: diagonal ABCD = two 1D chains (library 1D FFTs);
* brute force: stage matrices built element by element at 8x8;
* invariants: unitarity of L (Sec. 6.B), exact reversibility (Sec. 4.D),
  the factor product of Eq. Bnonsym08;
* the paper's printed error figures (Sec. 5.A, 5.B, 5.C);
* the direct method of Eq. Intro32 against the closed-form NsLCT of a Gaussian.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I
from tests.golden.loader import paper_matrices, paper_values

PM = paper_matrices()
PV = paper_values()


def _abcd(a, b, c, d):
    return np.block([[np.asarray(a, float), np.asarray(b, float)], [np.asarray(c, float), np.asarray(d, float)]])


EYE = np.eye(2)
ZERO = np.zeros((2, 2))
DFT_M = _abcd(ZERO, EYE, -EYE, ZERO)     # Eq. BasicDFT04, 2D FT
IDFT_M = _abcd(ZERO, -EYE, EYE, ZERO)    # Eq. BasicDFT04, 2D IFT


def _centered_fft2(g, inverse=False):
    """Library DFT over centred indices: sum_m e^{-+j2pi pm/N} g[m] with m, p centred."""
    x = np.fft.ifftshift(g)
    y = np.fft.ifft2(x) * g.size if inverse else np.fft.fft2(x)
    return np.fft.fftshift(y)


def _feasible_h(m, s, t):
    """A symmetric H on the feasible plane of m, offset (s, t) in the plane."""
    r, rhs = O.feasible_plane(m)
    rn = np.linalg.norm(r)
    h0 = r * rhs / rn ** 2
    _, _, vt = np.linalg.svd(r.reshape(1, 3))
    v = h0 + s * vt[1] + t * vt[2]
    return np.array([[v[0], v[1]], [v[1], v[2]]])


# ---------------------------------------------------------------- inputs


def test_random_symplectic_generator_is_symplectic():
    for seed in range(20):
        m = I.random_symplectic_abcd(seed)
        assert O.symplectic_residual(m) < 1e-14
        assert abs(np.linalg.det(m[:2, 2:])) >= 0.1


def test_hermite_gaussian_matches_library_hermite():
    from scipy.special import eval_hermite
    x = np.linspace(-6, 6, 301)
    for k in (0, 1, 2, 3, 11, 14, 18):
        ref = (2.0 ** k * math.factorial(k) * math.sqrt(math.pi)) ** -0.5 * np.exp(-x * x / 2) * eval_hermite(k, x)
        np.testing.assert_allclose(I.hermite_gaussian_1d(k, x), ref, rtol=1e-10, atol=1e-13)


# ---------------------------------------------------------------- ABCD handling


def test_printed_matrices_are_nearly_symplectic_and_project_exactly():
    expected_resid = {"M1": 1.7e-4, "M2": 4.5e-5, "M3": 9.9e-4, "M4": 6.1e-5, "MSELF": 6.3e-5}
    for name, m in PM.items():
        res = O.symplectic_residual(m)
        assert res == pytest.approx(expected_resid[name], rel=0.05), name
        p = O.project_sp4(m)
        assert O.symplectic_residual(p) < 1e-15 * max(1.0, np.max(np.abs(m)) ** 2), name
        # the clean-up moves the print by no more than its own constraint violation
        assert np.max(np.abs(p - m)) < 10 * res, name


def test_projection_keeps_symplectic_matrices():
    for seed in range(5):
        m = I.random_symplectic_abcd(100 + seed)
        np.testing.assert_allclose(O.project_sp4(m), m, atol=1e-14)


def test_feasible_plane_reproduces_lc_closed_forms():
    # Eq. LC08/LC10 are the one-parameter solutions of r.h = rhs
    for seed in range(10):
        m = I.random_symplectic_abcd(200 + seed)
        a, b, _, _ = O.split_abcd(m)
        r, rhs = O.feasible_plane(m)
        hx = (b[1, 0] - b[0, 1]) / a[1, 0]
        hy = (b[0, 1] - b[1, 0]) / a[0, 1]
        assert r @ np.array([hx, 0, 0]) == pytest.approx(rhs, abs=1e-12)
        assert r @ np.array([0, 0, hy]) == pytest.approx(rhs, abs=1e-12)
        for h in (np.diag([hx, 0.0]), np.diag([0.0, hy])):
            bp = b - a @ h
            assert abs(bp[0, 1] - bp[1, 0]) < 1e-12


def test_decomposition_product_equals_abcd():
    # Eq. Bnonsym08: (I,0;C1,I)(I,B';0,I)(I,0;C2,I)(I,H;0,I) = (A,B;C,D)
    mats = [O.project_sp4(m) for m in PM.values()] + [I.random_symplectic_abcd(300 + s) for s in range(8)]
    for m in mats:
        p = O.plan(m)
        np.testing.assert_allclose(O.compose_factors(p), m, atol=1e-12)
        assert p["Bp_asym"] < 1e-12 and p["C_asym"] < 1e-10
        assert abs(np.linalg.det(p["Bp"])) >= O.DET_FLOOR


def test_ha_search_is_no_worse_than_lc_or_random_feasible_points():
    rng = np.random.default_rng(7)
    for m in [O.project_sp4(PM["M1"]), O.project_sp4(PM["M2"])] + [I.random_symplectic_abcd(400 + s) for s in range(4)]:
        h = O.ha_search(m)
        best = O.ha_objective(m, h)
        hl = O.lc_h(m)
        if hl is not None:
            assert best <= O.ha_objective(m, hl) * (1 + 1e-9)
        for _ in range(50):
            hr = _feasible_h(m, *rng.uniform(-3, 3, size=2))
            if abs(np.linalg.det(O.decompose(m, hr)["Bp"])) < O.DET_FLOOR:
                continue
            assert best <= O.ha_objective(m, hr) * (1 + 1e-9)


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 16), (12, 8), (6, 10)])
def test_dft_special_case_equals_library_dft(nx, ny):
    """(0,I;-I,0) gives F of Eq. BasicDFT16 exactly when dx^2 = 2pi/Nx, dy^2 = 2pi/Ny
    and N is even, for any feasible H (the H only changes the route)."""
    dx, dy = I.default_spacing(nx), I.default_spacing(ny)
    g = I.blob_field(nx, ny, seed=nx * 100 + ny, width_range=(1.0, 3.0))
    ref = (dx * dy / (2j * math.pi)) * _centered_fft2(g)
    # A = 0, so every symmetric H is feasible (B' = I)
    for h in (None, np.array([[0.7, -0.4], [-0.4, 0.2]]), np.array([[-1.3, 0.9], [0.9, 0.5]])):
        out = O.forward(g, O.plan(DFT_M, h=h), dx, dy)
        assert O.rel_l2(out, ref) < 1e-13
    # (0,-I;I,0) gives the 2D IDFT exactly, with the constant dx dy / (-j 2pi):
    # the product of two 1D kernels with principal roots, 1/sqrt(-j2pi)^2. The
    # paper's 2D constant 1/(2pi sqrt(-det B)) with the principal root of -1
    # prints 1/(j 2pi) (Eq. BasicDFT20); the two differ by the global sign that
    # the metaplectic representation leaves free (it does not depend on H).
    # Exactness here holds for diagonal H (a non-diagonal h12 term meets the
    # unpaired Nyquist index -N/2 of the centred range); the DFT case above is
    # exact for every H.
    ref_i = (dx * dy / (-2j * math.pi)) * _centered_fft2(g, inverse=True)
    for h in (None, np.diag([0.7, -0.4]), np.diag([-1.5, -2.0])):
        out_i = O.forward(g, O.plan(IDFT_M, h=h), dx, dy)
        assert O.rel_l2(out_i, ref_i) < 1e-13


def test_dft_special_case_fails_for_odd_n():
    # the discrete chain only reaches the DFT exactly for even N (a property of the
    # centred frequency range, recorded so that a change in index origin is caught)
    n = 9
    d = I.default_spacing(n)
    g = I.blob_field(n, n, seed=5, width_range=(1.0, 3.0))
    ref = (d * d / (2j * math.pi)) * _centered_fft2(g)
    assert O.rel_l2(O.forward(g, O.plan(DFT_M), d, d), ref) > 0.1


def test_identity_and_cc_zero():
    g = I.blob_field(12, 10, seed=11)
    d = 0.37
    # A = I, B = 0: every invertible symmetric H is feasible (B' = -H)
    for h in (np.diag([0.8, -0.5]), np.array([[1.0, 0.3], [0.3, 2.0]])):
        out = O.forward(g, O.plan(np.eye(4), h=h), d, d)
        np.testing.assert_allclose(out, g, atol=1e-12)
    # CC^0 = F^-1 F = -I (constant (dx dy)(du dv)/(j 2pi)^2 * N^2 = -1)
    np.testing.assert_allclose(O.cc(g, np.zeros((2, 2)), d, 0.5), -g, atol=1e-12)


def test_pure_chirp_multiplication():
    c = np.array([[0.31, -0.22], [-0.22, 0.47]])
    m = _abcd(EYE, ZERO, c, EYE)  # Eq. BasicCM04
    nx, ny, dx, dy = 10, 14, 0.4, 0.3
    g = I.blob_field(nx, ny, seed=3)
    p = np.arange(nx)[:, None] - nx // 2
    q = np.arange(ny)[None, :] - ny // 2
    ref = g * np.exp(0.5j * (c[0, 0] * (p * dx) ** 2 + 2 * c[0, 1] * (p * dx) * (q * dy) + c[1, 1] * (q * dy) ** 2))
    out = O.forward(g, O.plan(m, h=np.array([[1.2, 0.1], [0.1, -0.9]])), dx, dy)
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_pure_chirp_convolution_equals_library_fft_convolution():
    """(I,B;0,I) with B symmetric: the chain CC^{B-H} CC^{H} = -CC^{B}, i.e.
    ifft2(chi_B * fft2(g)) with chi_B(k) = exp(-j/2 k^T B k) at the DFT's
    frequency spacing 2 pi/(N d) (library FFT, centred bins)."""
    b = np.array([[0.9, 0.35], [0.35, -0.6]])
    m = _abcd(EYE, b, ZERO, EYE)
    nx, ny = 16, 12
    dx, dy = 0.5, 0.45
    g = I.blob_field(nx, ny, seed=21)
    kx = (np.arange(nx) - nx // 2)[:, None] * (2 * math.pi / (nx * dx))
    ky = (np.arange(ny) - ny // 2)[None, :] * (2 * math.pi / (ny * dy))
    chi = np.exp(-0.5j * (b[0, 0] * kx * kx + 2 * b[0, 1] * kx * ky + b[1, 1] * ky * ky))
    ref = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(chi) * np.fft.fft2(np.fft.ifftshift(g))))
    out = O.forward(g, O.plan(m), dx, dy)
    np.testing.assert_allclose(out, ref, atol=1e-12)


def _chain_1d(x, a, b, c, d, h, delta, axis):
    """1D CM-CC-CM-CC chain along one axis with library FFTs: the 1D analogue of
    Eq. HA28 with constants delta/sqrt(j 2pi) (F) and dw/sqrt(j 2pi) (F^-1)."""
    n = x.shape[axis]
    dw = 2 * math.pi / (n * delta)
    s = np.sqrt(2j * math.pi)
    idx = np.arange(n) - n // 2
    shape = [1, 1]
    shape[axis] = n
    idx = idx.reshape(shape)

    def cm1(y, cc_, dl):
        return y * np.exp(0.5j * cc_ * (idx * dl) ** 2)

    def f1(y, sign, dl):
        yy = np.fft.ifftshift(y, axes=axis)
        yy = np.fft.fft(yy, axis=axis) if sign < 0 else np.fft.ifft(yy, axis=axis) * n
        return (dl / s) * np.fft.fftshift(yy, axes=axis)

    def cc1(y, bb):
        return f1(cm1(f1(y, -1, delta), -bb, dw), +1, dw)

    bp = b - a * h
    dp = d - c * h
    c2 = (a - 1.0) / bp
    c1 = (dp - 1.0) / bp
    return cm1(cc1(cm1(cc1(x, h), c2, delta), bp), c1, delta)


def test_separable_abcd_equals_two_1d_chains():
    # two 1D symplectic (a, b; c, d) with ad - bc = 1, one per axis (Sec. 1: the
    # separable LCT is a special case of the NsLCT)
    ax_, bx_, cx_ = 0.8, 1.1, -0.3
    dx_ = (1 + bx_ * cx_) / ax_
    ay_, by_, cy_ = -0.6, 0.7, 0.9
    dy_ = (1 + by_ * cy_) / ay_
    m = _abcd(np.diag([ax_, ay_]), np.diag([bx_, by_]), np.diag([cx_, cy_]), np.diag([dx_, dy_]))
    assert O.symplectic_residual(m) < 1e-14
    hx, hy = 0.45, -0.8
    nx, ny = 12, 16
    delx, dely = 0.55, 0.4
    g = I.blob_field(nx, ny, seed=8)
    ref = _chain_1d(_chain_1d(g, ax_, bx_, cx_, dx_, hx, delx, 0), ay_, by_, cy_, dy_, hy, dely, 1)
    out = O.forward(g, O.plan(m, h=np.diag([hx, hy])), delx, dely)
    np.testing.assert_allclose(out, ref, atol=1e-12)


# ---------------------------------------------------------------- brute force / invariants


def _dense_stage_matrices(nx, ny, params, dx, dy):
    """Stage matrices of Eq. self12 built entry by entry with Python loops."""
    n2 = nx * ny
    dwx, dwy = 2 * math.pi / (nx * dx), 2 * math.pi / (ny * dy)

    def idx(i, j):
        return i * ny + j

    def cm_mat(c, du, dv):
        mat = np.zeros((n2, n2), dtype=complex)
        for i in range(nx):
            for j in range(ny):
                p, q = (i - nx // 2) * du, (j - ny // 2) * dv
                mat[idx(i, j), idx(i, j)] = np.exp(0.5j * (c[0, 0] * p * p + (c[0, 1] + c[1, 0]) * p * q + c[1, 1] * q * q))
        return mat

    def dft_mat(sign, du, dv):
        mat = np.zeros((n2, n2), dtype=complex)
        for i in range(nx):
            for j in range(ny):
                for k in range(nx):
                    for l in range(ny):
                        p, q, mm, nn = i - nx // 2, j - ny // 2, k - nx // 2, l - ny // 2
                        mat[idx(i, j), idx(k, l)] = np.exp(sign * 2j * math.pi * (p * mm / nx + q * nn / ny))
        return (du * dv / (2j * math.pi)) * mat

    f = dft_mat(-1, dx, dy)
    fi = dft_mat(+1, dwx, dwy)
    cc_h = fi @ cm_mat(-params["H"], dwx, dwy) @ f
    cc_b = fi @ cm_mat(-params["Bp"], dwx, dwy) @ f
    return cm_mat(params["C1"], dx, dy) @ cc_b @ cm_mat(params["C2"], dx, dy) @ cc_h


def _dense_from_operator(op, nx, ny):
    n2 = nx * ny
    mat = np.zeros((n2, n2), dtype=complex)
    for k in range(n2):
        e = np.zeros(n2, dtype=complex)
        e[k] = 1.0
        mat[:, k] = op(e.reshape(nx, ny)).reshape(-1)
    return mat


def test_brute_force_stage_matrices_8x8_and_unitarity():
    nx = ny = 8
    m = I.random_symplectic_abcd(1234)
    params = O.plan(m)
    d = I.default_spacing(8)
    dense = _dense_stage_matrices(nx, ny, params, d, d)
    lmat = _dense_from_operator(lambda x: O.forward(x, params, d, d), nx, ny)
    np.testing.assert_allclose(lmat, dense, atol=1e-12)
    # Sec. 6.B: L is unitary
    np.testing.assert_allclose(lmat.conj().T @ lmat, np.eye(64), atol=1e-12)
    # the exact inverse chain is L^H
    linv = _dense_from_operator(lambda x: O.inverse(x, params, d, d), nx, ny)
    np.testing.assert_allclose(linv, lmat.conj().T, atol=1e-12)


def test_unitarity_nonsquare_other_spacing():
    nx, ny = 6, 8
    m = O.project_sp4(PM["M2"])
    params = O.plan(m)
    lmat = _dense_from_operator(lambda x: O.forward(x, params, 0.3, 0.7), nx, ny)
    np.testing.assert_allclose(lmat.conj().T @ lmat, np.eye(nx * ny), atol=1e-12)


def test_exact_reversibility():
    # Sec. 4.D / 5.C: forward then the inverse chain returns the input exactly;
    # the paper reports ~279 dB PSNR (FP64 round-off)
    for seed, (nx, ny) in enumerate([(64, 64), (48, 40), (100, 100)]):
        m = I.random_symplectic_abcd(500 + seed)
        params = O.plan(m)
        g = I.blob_field(nx, ny, seed=seed)
        d = I.default_spacing(nx)
        back = O.inverse(O.forward(g, params, d, d), params, d, d)
        err = O.nmse(back, g)
        assert err < 1e-25
        psnr = 10 * math.log10(np.max(np.abs(g)) ** 2 / np.mean(np.abs(back - g) ** 2))
        assert psnr > 0.8 * PV["psnr_rev_db"]


# ---------------------------------------------------------------- direct method (Eq. Intro32)


def _gaussian_nslct(m, u, v):
    """Closed-form NsLCT (Eq. Intro08) of g(x, y) = exp(-(x^2 + y^2)/2)."""
    a, b, c, d = O.split_abcd(m)
    bi = np.linalg.inv(b)
    s = O.sym_part(bi @ a)
    q = np.eye(2) - 1j * s
    sig = np.linalg.eigvalsh(s)
    sqrt_det_q = np.prod(np.sqrt(1 - 1j * sig))  # each factor has Re > 0
    qi = np.linalg.inv(q)
    dbi = O.sym_part(d @ bi)
    out = np.empty((len(u), len(v)), dtype=complex)
    for i, uu in enumerate(u):
        for j, vv in enumerate(v):
            zp = np.array([uu, vv])
            bl = -1j * (bi @ zp)
            out[i, j] = np.exp(0.5j * zp @ dbi @ zp + 0.5 * bl @ qi @ bl)
    return out / (np.sqrt(complex(-np.linalg.det(b))) * sqrt_det_q)


@pytest.mark.parametrize("name", ["M2", "M4", "rand"])
def test_direct_method_matches_closed_form_gaussian(name):
    m = I.random_symplectic_abcd(77) if name == "rand" else O.project_sp4(PM[name])
    n, delta = 160, 0.1
    x = (np.arange(n) - n // 2) * delta
    g = np.exp(-0.5 * (x[:, None] ** 2 + x[None, :] ** 2))
    du = 0.35
    out = O.direct(g, m, delta, delta, du, du, 12, 12)
    u = (np.arange(12) - 6) * du
    ref = _gaussian_nslct(m, u, u)
    assert O.rel_l2(out, ref) < 1e-8


# ---------------------------------------------------------------- the paper's printed figures


@pytest.fixture(scope="module")
def reference_outputs():
    """Direct-method references on the paper's fine grid (1024^2, delta 0.078, Sec. 5.A)."""
    n_ref = int(PV["ref_grid_n"])
    d_ref = PV["ref_grid_delta"]
    m1 = O.project_sp4(PM["M1"])
    m2 = O.project_sp4(PM["M2"])
    g1_fine = I.hg_field([(1, 2), (3, 1)], n_ref, d_ref)
    g2_fine = I.hg_field([(2, 18), (14, 11)], n_ref, d_ref)
    return {
        "g1": O.direct(g1_fine, m1, d_ref, d_ref, 0.25, 0.25, 100, 100),
        "g2": O.direct(g2_fine, m2, d_ref, d_ref, 0.2, 0.2, 165, 165),
    }


@pytest.mark.slow
@pytest.mark.parametrize("method", ["ha", "lc"])
def test_printed_accuracy(reference_outputs, method):
    m1 = O.project_sp4(PM["M1"])
    m2 = O.project_sp4(PM["M2"])
    g1 = I.hg_field([(1, 2), (3, 1)], 100, 0.25)
    g2 = I.hg_field([(2, 18), (14, 11)], 165, 0.2)
    e1 = O.nmse(O.transform(g1, m1, 0.25, 0.25, method=method), reference_outputs["g1"])
    e2 = O.nmse(O.transform(g2, m2, 0.2, 0.2, method=method), reference_outputs["g2"])
    for got, key in ((e1, f"nmse_acc_g1_M1_{method}"), (e2, f"nmse_acc_g2_M2_{method}")):
        assert PV[key] / 1.5 < got < PV[key] * 1.5, (key, got)


@pytest.mark.parametrize("method", ["ha", "lc"])
def test_printed_additivity(method):
    cases = [
        ("g1", [(1, 2), (3, 1)], 100, 0.25, "M1", "M3"),
        ("g2", [(2, 18), (14, 11)], 165, 0.2, "M2", "M4"),
    ]
    for gname, terms, n, d, first, second in cases:
        ma = O.project_sp4(PM[first])
        mb = O.project_sp4(PM[second])
        g = I.hg_field(terms, n, d)
        two = O.transform(O.transform(g, ma, d, d, method=method), mb, d, d, method=method)
        one = O.transform(g, mb @ ma, d, d, method=method)
        key = f"nmse_add_{gname}_{second}{first}_{method}"
        got = O.nmse(one, two)
        assert PV[key] / 1.5 < got < PV[key] * 1.5, (key, got)


# ---------------------------------------------------------------- zero padding (Secs. 2.A, 5.A)


def test_zero_padding_geometry_and_reversibility():
    m = I.random_symplectic_abcd(91)
    params = O.plan(m)
    g = I.blob_field(10, 14, seed=91)
    d = 0.6
    # dN = 0 is the plain chain
    np.testing.assert_array_equal(O.forward_padded(g, params, d, d, 10, 14), O.forward(g, params, d, d))
    # placement keeps centred indices: the field's centre sample stays the grid's centre
    gp = O.zero_pad(g, 16, 24)
    assert gp[8, 12] == g[5, 7] and np.count_nonzero(gp) == np.count_nonzero(g)
    np.testing.assert_array_equal(O.centre_crop(gp, 10, 14), g)
    # the padded chain is still exactly invertible, zeros included
    full = O.forward_padded(g, params, d, d, 16, 24)
    assert full.shape == (16, 24)
    back = O.inverse(full, params, d, d)
    assert np.max(np.abs(back - gp)) < 1e-12
    np.testing.assert_allclose(O.inverse_padded(full, params, d, d, 16, 24, 10, 14), g, atol=1e-12)
    # the cropped output is the centre of the full one
    np.testing.assert_array_equal(O.forward_padded(g, params, d, d, 16, 24, crop=True), O.centre_crop(full, 10, 14))


def test_zero_padding_reduces_aliasing(reference_outputs):
    """Sec. 5.A: g2 under M2 spreads beyond its 165 x 165 window and aliases
    (NMSE 1.1e-3, printed); zero-padding the input to (165 + dN)^2 removes
    it: against the direct method (Eq. Intro32) on each padded output grid the
    NMSE falls below 1e-5 at dN = 20 and below 1e-6 at dN = 50."""
    n_ref = int(PV["ref_grid_n"])
    d_ref = PV["ref_grid_delta"]
    m2 = O.project_sp4(PM["M2"])
    g2 = I.hg_field([(2, 18), (14, 11)], 165, 0.2)
    g2_fine = I.hg_field([(2, 18), (14, 11)], n_ref, d_ref)
    params = O.plan(m2)
    errs = [O.nmse(O.forward(g2, params, 0.2, 0.2), reference_outputs["g2"])]
    for dn in (20, 50):
        n = 165 + dn
        ref = O.direct(g2_fine, m2, d_ref, d_ref, 0.2, 0.2, n, n)
        errs.append(O.nmse(O.forward_padded(g2, params, 0.2, 0.2, n, n), ref))
    assert errs[0] > 5e-4
    assert errs[1] < 1e-5 and errs[2] < 1e-6
    assert errs[0] > errs[1] > errs[2]


# ---------------------------------------------------------------- filtering in two NsLCT domains (Sec. 5.B)


def test_filter_pipelines_all_pass_identities():
    """All-pass filters: Eq. Add04 returns the input exactly (each inverse is
    exact), and since every chain is unitary the deviation of Eq. Add08 from
    the input equals the additivity error of Eq. Add16 exactly."""
    m1, m3 = I.random_symplectic_abcd(31), I.random_symplectic_abcd(32)
    p1, p3, p31 = O.plan(m1), O.plan(m3), O.plan(m3 @ m1)
    n, d = 24, float(np.sqrt(2 * np.pi / 24))
    g = I.blob_field(n, n, seed=33, width_range=(1.5, 3.0))
    ones = np.ones((n, n))
    back = O.filter_two_domains(g, p1, p3, ones, ones, d, d)
    assert np.max(np.abs(back - g)) < 1e-12
    g8 = O.filter_two_domains_additive(g, p1, p3, p31, ones, ones, d, d)
    e_add = O.nmse_add(g, p1, p3, p31, d, d)
    assert e_add > 1e-8
    assert abs(O.nmse(g8, g) - e_add) < 1e-9 * e_add


def test_filter_pipelines_differ_by_the_additivity_error():
    """With real filters the two pipelines differ by at most what the
    additivity error allows: ||Add08 - Add04|| <= ||h3|| sqrt(NMSE_add-like)
    (the composed inverse replaces two inverses; both unitary)."""
    m1, m3 = O.project_sp4(PM["M1"]), O.project_sp4(PM["M3"])
    p1, p3, p31 = O.plan(m1), O.plan(m3), O.plan(m3 @ m1)
    g = I.hg_field([(1, 2), (3, 1)], 100, 0.25)
    h1 = I.gaussian_mask(100, 100, 0.3, tilt=2.0)
    h3 = I.gaussian_mask(100, 100, 0.4)
    a = O.filter_two_domains(g, p1, p3, h1, h3, 0.25, 0.25)
    b = O.filter_two_domains_additive(g, p1, p3, p31, h1, h3, 0.25, 0.25)
    # Add08 - Add04 = (L31^-1 - L1^-1 L3^-1) y with y = h3 L3 h1 L1 g, and
    # L31^-1 - L1^-1 L3^-1 = L31^-1 (I - L31 L1^-1 L3^-1): small when additive
    y = h3 * O.forward(h1 * O.forward(g, p1, 0.25, 0.25), p3, 0.25, 0.25)
    z = O.inverse(O.inverse(y, p3, 0.25, 0.25), p1, 0.25, 0.25)
    rel = np.linalg.norm(O.forward(z, p31, 0.25, 0.25) - y) / np.linalg.norm(y)
    assert abs(np.linalg.norm(b - a) / np.linalg.norm(y) - rel) < 1e-10
    assert rel < 0.05


# ---------------------------------------------------------------- CC-CM-CC-CM decomposition (Sec. 4.C)


def test_type2_decomposition_identities():
    """Eq. CCCMCCCM16's factors multiply back to M; by Eqs. CCCMCCCM20-30 the
    type-2 chain of M^-1 with H1 = -H is the type-1 inverse chain of M; the
    type-2 criterion of M at H1 is the type-1 criterion of M^-1 at -H1; the
    chain is exactly reversible and reduces to the 2D DFT of Eq. BasicDFT16."""
    n = 16
    d = float(np.sqrt(2 * np.pi / n))
    g = I.blob_field(n, n, seed=8, width_range=(1.5, 3.0))
    for s in range(3):
        m = I.random_symplectic_abcd(80 + s)
        p2 = O.plan_type2(m)
        assert p2["Bp1_asym"] < 1e-12
        assert np.max(np.abs(O.compose_factors_type2(p2) - m)) < 1e-12
        mi = O.symplectic_inverse(m)
        assert np.max(np.abs(mi @ m - np.eye(4))) < 1e-12
        assert abs(O.ha_objective_type2(m, p2["H1"]) - O.ha_objective(mi, -p2["H1"])) < 1e-9
        p1 = O.plan(m)
        dual = O.forward_type2(g, O.decompose_type2(mi, -p1["H"]), d, d)
        assert np.max(np.abs(dual - O.inverse(g, p1, d, d))) < 1e-12
        back = O.inverse_type2(O.forward_type2(g, p2, d, d), p2, d, d)
        assert np.max(np.abs(back - g)) < 1e-12
    z, e = np.zeros((2, 2)), np.eye(2)
    dft = np.block([[z, e], [-e, z]])
    out = O.forward_type2(g, O.plan_type2(dft), d, d)
    ref = d * d / (2j * np.pi) * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(g)))
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


def test_trace_rule():
    """Eq. Reversible08 picks type 2 exactly when tr(B) < 0; M and M^-1 have
    opposite traces of B, so forward and inverse use different types."""
    for s in range(6):
        m = I.random_symplectic_abcd(90 + s)
        tb = np.trace(m[:2, 2:])
        assert O.uses_type2(m) == (tb < 0)
        if tb != 0:
            assert O.uses_type2(O.symplectic_inverse(m)) != O.uses_type2(m)


@pytest.mark.parametrize("phi", [0.4, 1.1])
def test_fractional_fourier_case_has_hermite_gaussian_eigenfunctions(phi):
    """For M = (cos phi I, sin phi I; -sin phi I, cos phi I) the NsLCT is the 2D
    fractional Fourier transform, whose eigenfunctions are the Hermite-Gaussians
    HG_{k,l} (Eq. Acc16) with eigenvalues exp(-j (k + l + 1) phi). Under the
    sampling condition the chain reproduces both, global phase included."""
    n = 64
    d = float(np.sqrt(2 * np.pi / n))
    c, s = np.cos(phi), np.sin(phi)
    e = np.eye(2)
    m = np.block([[c * e, s * e], [-s * e, c * e]])
    for k, l in [(0, 0), (1, 2), (3, 1), (2, 5)]:
        g = I.hg_field([(k, l)], n, d)
        out = O.transform(g, m, d, d)
        lam = np.exp(-1j * (k + l + 1) * phi)
        assert np.linalg.norm(out - lam * g) < 1e-12 * np.linalg.norm(g), (k, l)
