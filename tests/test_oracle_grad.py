"""Pins for the oracle's gradients (the adjoint of Eq. HA28 and the 10-parameter
ABCD parametrisation): checked against central finite differences of the
oracle's forward transform in FP64, and against the exact inverse chain
(L is unitary, Sec. 6.B, so L^H = L^-1)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I


def test_theta_round_trip_and_symplectic():
    for seed in range(8):
        m = I.random_symplectic_abcd(600 + seed)
        th = O.theta_from_abcd(m)
        np.testing.assert_allclose(O.abcd_from_theta(th), m, atol=1e-13)
        rng = np.random.default_rng(seed)
        m2 = O.abcd_from_theta(th + 0.1 * rng.standard_normal(10))
        assert O.symplectic_residual(m2) < 1e-13


def test_h_rule_is_feasible_and_fixes_feasible_h():
    m = I.random_symplectic_abcd(610)
    h0 = O.ha_search(m)
    th = O.theta_from_abcd(m)
    np.testing.assert_allclose(O.h_of_theta(th, h0), h0, atol=1e-13)
    th2 = th + 0.05 * np.arange(1, 11) / 10
    h2 = O.h_of_theta(th2, h0)
    r, rhs = O.feasible_plane(O.abcd_from_theta(th2))
    assert abs(r @ np.array([h2[0, 0], h2[0, 1], h2[1, 1]]) - rhs) < 1e-12


def test_complex_step_jacobian_matches_finite_differences():
    m = I.random_symplectic_abcd(611)
    h0 = O.ha_search(m)
    th = O.theta_from_abcd(m)
    jac = O.chirp_jacobian(th, h0)
    eps = 1e-6
    fd = np.stack([(O._chirp_vec(th + eps * np.eye(10)[k], h0) - O._chirp_vec(th - eps * np.eye(10)[k], h0)) / (2 * eps)
                   for k in range(10)], axis=1)
    np.testing.assert_allclose(jac, fd, atol=1e-7 * max(1.0, np.max(np.abs(fd))))


@pytest.mark.parametrize("nx,ny", [(16, 16), (12, 16)])
def test_parameter_gradient_matches_finite_differences(nx, ny):
    m = I.random_symplectic_abcd(612 + nx)
    h0 = O.ha_search(m)
    dx, dy = I.default_spacing(nx), I.default_spacing(ny)
    x = I.blob_field(nx, ny, seed=1, width_range=(1, 3))
    yt = I.blob_field(nx, ny, seed=2, width_range=(1, 3))
    loss, gx, gth, gch = O.loss_and_grad(x, yt, m, h0, dx, dy)
    th = O.theta_from_abcd(m)

    def lossf(t):
        p = O.params_from_theta(t, h0)
        return float(np.sum(np.abs(O.forward(x, p, dx, dy) - yt) ** 2))

    eps = 1e-6
    fd = np.array([(lossf(th + eps * np.eye(10)[k]) - lossf(th - eps * np.eye(10)[k])) / (2 * eps) for k in range(10)])
    np.testing.assert_allclose(gth, fd, rtol=1e-6, atol=1e-7 * np.max(np.abs(fd)))
    assert loss == pytest.approx(lossf(th), rel=1e-12)


def test_chirp_gradient_matches_finite_differences():
    # perturb each chirp entry of a fixed decomposition directly
    nx = ny = 16
    m = I.random_symplectic_abcd(620)
    p0 = O.plan(m)
    d = I.default_spacing(nx)
    x = I.blob_field(nx, ny, seed=3, width_range=(1, 3))
    yt = I.blob_field(nx, ny, seed=4, width_range=(1, 3))
    r = O.forward(x, p0, d, d) - yt
    _, gch = O.chain_vjp(x, 2 * r, p0, d, d)
    names = ["H", "Bp", "C1", "C2"]
    eps = 1e-6
    for s, name in enumerate(names):
        for k, (i, j) in enumerate([(0, 0), (0, 1), (1, 1)]):
            e = np.zeros((2, 2))
            e[i, j] = e[j, i] = 1.0
            pp = dict(p0); pm = dict(p0)
            pp[name] = p0[name] + eps * e
            pm[name] = p0[name] - eps * e
            lp = np.sum(np.abs(O.forward(x, pp, d, d) - yt) ** 2)
            lm = np.sum(np.abs(O.forward(x, pm, d, d) - yt) ** 2)
            assert gch[3 * s + k] == pytest.approx((lp - lm) / (2 * eps), rel=1e-6, abs=1e-6)


def test_input_gradient_is_inverse_chain_and_matches_fd():
    nx, ny = 12, 16
    m = I.random_symplectic_abcd(630)
    h0 = O.ha_search(m)
    dx, dy = I.default_spacing(nx), I.default_spacing(ny)
    x = I.blob_field(nx, ny, seed=5, width_range=(1, 3))
    yt = I.blob_field(nx, ny, seed=6, width_range=(1, 3))
    loss, gx, _, _ = O.loss_and_grad(x, yt, m, h0, dx, dy)
    p = O.params_from_theta(O.theta_from_abcd(m), h0)
    gbar = 2 * (O.forward(x, p, dx, dy) - yt)
    np.testing.assert_allclose(gx, O.inverse(gbar, p, dx, dy), atol=1e-12 * np.max(np.abs(gx)))
    eps = 1e-6
    for (i, j) in [(0, 0), (5, 7), (11, 15)]:
        e = np.zeros_like(x)
        e[i, j] = 1.0

        def lx(z):
            return float(np.sum(np.abs(O.forward(z, p, dx, dy) - yt) ** 2))
        fr = (lx(x + eps * e) - lx(x - eps * e)) / (2 * eps)
        fi = (lx(x + 1j * eps * e) - lx(x - 1j * eps * e)) / (2 * eps)
        assert gx[i, j] == pytest.approx(fr + 1j * fi, rel=1e-6, abs=1e-8)
