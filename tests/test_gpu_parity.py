"""GPU parity: the CUDA chain (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs, with the plan's own H fed to the
oracle (so near-ties in the H criterion cannot break parity).

Tolerances (relative L2 over the whole field):
* FP32 (complex64) path: 2e-5;
* FP64 (complex128) path: 1e-12 at N <= 64, growing linearly with N above.
  Both sides round chirp phases of magnitude ~ |c| (N/2)^2 dx^2 / 2, which is
  ~ |c| pi N / 4 under the sampling condition dx^2 = 2 pi / N, so their FP64
  rounding differences grow in proportion to N.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I
from tests.golden.loader import paper_matrices

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL32 = 2e-5
TOL64 = 1e-12


def tol64(nx, ny):
    return TOL64 * max(1.0, max(nx, ny) / 64.0)
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


def _plan(N, m, nx, ny, precision="fp32", **kw):
    return N.Plan(m, nx, ny, precision=precision, **kw)


def _gpu(plan, g, inverse=False):
    dt = torch.complex128 if plan.dtype == torch.complex128 else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(g)).to(dt).cuda()
    y = plan.inverse(x) if inverse else plan.forward(x)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


def _oracle(plan, g, inverse=False):
    p = plan.params()
    info = plan.info()
    params = O.decompose(info["abcd"], p["H"])
    f = O.inverse if inverse else O.forward
    return f(g, params, plan.dx, plan.dy)


# ---------------------------------------------------------------- small FP64 case


def test_fp64_64x64_forward_inverse(N):
    """64x64 complex128, blob input, random symplectic ABCD (seed 0)."""
    m = I.random_symplectic_abcd(0)
    g = I.blob_field(64, 64, seed=0)
    plan = _plan(N, m, 64, 64, precision="fp64")
    out = _gpu(plan, g)
    ref = _oracle(plan, g)
    assert O.rel_l2(out, ref) < TOL64
    back = _gpu(plan, out, inverse=True)
    assert O.rel_l2(back, g) < TOL64
    np.testing.assert_allclose(back, _oracle(plan, out, inverse=True), atol=1e-12 * np.max(np.abs(g)))


# ---------------------------------------------------------------- 512^2 FP32


def test_fp32_512_blob(N):
    m = I.random_symplectic_abcd(1)
    g = I.blob_field(512, 512, seed=1)
    plan = _plan(N, m, 512, 512)
    out = _gpu(plan, g)
    ref = _oracle(plan, g)
    assert O.rel_l2(out, ref) < TOL32
    back = _gpu(plan, out, inverse=True)
    assert O.rel_l2(back, g) < TOL32


@pytest.mark.parametrize("case", ["dft", "idft", "identity", "separable", "pure_cm", "pure_cc"])
def test_fp32_512_special_cases(N, case):
    n = 512
    d = I.default_spacing(n)
    z, e = np.zeros((2, 2)), np.eye(2)
    if case == "dft":
        m = np.block([[z, e], [-e, z]])
    elif case == "idft":
        m = np.block([[z, -e], [e, z]])
    elif case == "identity":
        m = np.eye(4)
    elif case == "separable":
        ax, bx, cx = 0.8, 1.1, -0.3
        ay, by, cy = -0.6, 0.7, 0.9
        m = np.block([[np.diag([ax, ay]), np.diag([bx, by])],
                      [np.diag([cx, cy]), np.diag([(1 + bx * cx) / ax, (1 + by * cy) / ay])]])
    elif case == "pure_cm":
        m = np.block([[e, z], [np.array([[0.3, -0.2], [-0.2, 0.45]]), e]])
    else:
        m = np.block([[e, np.array([[0.9, 0.35], [0.35, -0.6]])], [z, e]])
    g = I.blob_field(n, n, seed=11)
    plan = _plan(N, m, n, n)
    out = _gpu(plan, g)
    ref = _oracle(plan, g)
    assert O.rel_l2(out, ref) < TOL32
    if case == "dft":
        lib_ref = (d * d / (2j * math.pi)) * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(g)))
        assert O.rel_l2(out, lib_ref) < TOL32
    if case == "identity":
        assert O.rel_l2(out, g) < TOL32


@pytest.mark.parametrize("name", ["M1", "M2", "M3", "M4", "MSELF"])
@pytest.mark.parametrize("method", ["ha", "lc"])
def test_fp32_paper_matrices(N, name, method):
    n = 256
    g = I.hg_field([(1, 2), (3, 1)], n, I.default_spacing(n))
    plan = _plan(N, PM[name], n, n, method=method, project=True)
    np.testing.assert_allclose(plan.info()["abcd"], O.project_sp4(PM[name]), atol=1e-12)
    out = _gpu(plan, g)
    assert O.rel_l2(out, _oracle(plan, g)) < TOL32


# ---------------------------------------------------------------- shapes, ragged panels, radix 3


SHAPES = [(8, 8), (12, 16), (16, 12), (48, 64), (64, 48), (96, 192), (192, 96), (384, 24),
          (24, 384), (768, 128), (128, 1536), (1536, 64), (2048, 32), (32, 4096), (256, 1024),
          (4096, 8), (8, 4096)]


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_fp32_shapes(N, nx, ny):
    seed = nx * 7 + ny
    m = I.random_symplectic_abcd(seed)
    g = I.blob_field(nx, ny, seed=seed, width_range=(1.0, max(2.0, min(nx, ny) / 8)))
    plan = _plan(N, m, nx, ny)
    out = _gpu(plan, g)
    assert O.rel_l2(out, _oracle(plan, g)) < TOL32
    inv = _gpu(plan, g, inverse=True)
    assert O.rel_l2(inv, _oracle(plan, g, inverse=True)) < TOL32


@pytest.mark.parametrize("nx,ny", [(8, 8), (12, 24), (96, 64), (256, 128)])
def test_fp64_shapes(N, nx, ny):
    m = I.random_symplectic_abcd(nx + ny)
    g = I.blob_field(nx, ny, seed=nx + 3 * ny, width_range=(1.0, 4.0))
    plan = _plan(N, m, nx, ny, precision="fp64")
    assert O.rel_l2(_gpu(plan, g), _oracle(plan, g)) < tol64(nx, ny)


def test_degenerate_plane_and_user_h(N):
    n = 128
    g = I.blob_field(n, n, seed=5)
    m = I.random_symplectic_abcd(9, middle="gyrator")  # r = 0: 3D H search
    plan = _plan(N, m, n, n)
    assert O.rel_l2(_gpu(plan, g), _oracle(plan, g)) < TOL32
    h = np.array([[0.4, -0.1], [-0.1, 0.7]])
    plan_u = _plan(N, m, n, n, h=h)
    np.testing.assert_allclose(plan_u.params()["H"], h, atol=0)
    assert O.rel_l2(_gpu(plan_u, g), _oracle(plan_u, g)) < TOL32


# ---------------------------------------------------------------- buffers, streams, determinism


def test_in_place_and_determinism(N):
    n = 256
    m = I.random_symplectic_abcd(21)
    g = torch.from_numpy(I.blob_field(n, n, seed=21)).to(torch.complex64).cuda()
    plan = _plan(N, m, n, n)
    a = plan.forward(g)
    b = plan.forward(g)
    x = g.clone()
    plan.forward(x, out=x)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(a, x)


def test_side_stream(N):
    n = 256
    m = I.random_symplectic_abcd(22)
    g = torch.from_numpy(I.blob_field(n, n, seed=22)).to(torch.complex64).cuda()
    plan = _plan(N, m, n, n)
    ref = plan.forward(g)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        out = plan.forward(g)
    torch.cuda.synchronize()
    assert torch.equal(ref, out)


def test_binding_validates_buffers(N):
    plan = _plan(N, I.random_symplectic_abcd(2), 64, 64)
    with pytest.raises(ValueError):
        plan.forward(torch.zeros(64, 64, dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):
        plan.forward(torch.zeros(64, 32, dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        plan.forward(torch.zeros(64, 64, dtype=torch.complex64))


# ---------------------------------------------------------------- full size (4096^2, the bench workload)


@pytest.fixture(scope="module")
def field_4096():
    g = I.add_white_noise(I.blob_field(4096, 4096, seed=2), sigma=0.05, seed=102)
    return g


def test_4096_properties(N, field_4096):
    """Properties that hold at any size: L is unitary (Sec. 6.B: norm kept)
    and exactly invertible (Sec. 4.D), checked on the bench workload."""
    x = torch.from_numpy(field_4096).to(torch.complex64).cuda()
    for k in range(3):
        plan = _plan(N, I.random_symplectic_abcd(200 + k), 4096, 4096)
        y = plan.forward(x)
        z = plan.inverse(y)
        torch.cuda.synchronize()
        nx_ = torch.linalg.vector_norm(x.to(torch.complex128)).item()
        ny_ = torch.linalg.vector_norm(y.to(torch.complex128)).item()
        assert abs(ny_ / nx_ - 1) < 1e-5
        err = torch.linalg.vector_norm((z - x).to(torch.complex128)).item() / nx_
        assert err < TOL32


def test_4096_dft_case_matches_library_fft(N, field_4096):
    n = 4096
    d = I.default_spacing(n)
    z, e = np.zeros((2, 2)), np.eye(2)
    plan = _plan(N, np.block([[z, e], [-e, z]]), n, n)
    out = _gpu(plan, field_4096)
    ref = (d * d / (2j * math.pi)) * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(field_4096)))
    assert O.rel_l2(out, ref) < TOL32


def test_4096_full_oracle(N, field_4096):
    """One full 4096^2 transform against the direct-sum oracle (FP64 dense DFTs)."""
    plan = _plan(N, I.random_symplectic_abcd(200), 4096, 4096)
    out = _gpu(plan, field_4096)
    ref = _oracle(plan, field_4096)
    assert O.rel_l2(out, ref) < TOL32


def test_zero_field_gives_exact_zeros(N):
    """The chain is linear: a zero field maps to exact zeros (no NaN from the
    chirps or the twiddle powers), in every precision."""
    for precision, dt in (("fp32", torch.complex64), ("fp64", torch.complex128), ("mixed", torch.complex64)):
        plan = _plan(N, I.random_symplectic_abcd(3), 256, 512, precision=precision)
        x = torch.zeros(256, 512, dtype=dt, device="cuda")
        y = plan.forward(x)
        z = plan.inverse(x)
        torch.cuda.synchronize()
        assert int(torch.count_nonzero(y)) == 0 and int(torch.count_nonzero(z)) == 0


def test_fp64_4096_full_oracle(N, field_4096):
    """The largest size in complex128 against the direct-sum oracle."""
    plan = _plan(N, I.random_symplectic_abcd(201), 4096, 4096, precision="fp64")
    out = _gpu(plan, field_4096)
    ref = _oracle(plan, field_4096)
    assert O.rel_l2(out, ref) < tol64(4096, 4096)


@pytest.mark.parametrize("n", [256, 4096])
def test_bounded_wait_expires_and_plan_recovers(N, n):
    """Failure detection without a fault: a pass whose barriers can never
    complete gives up after 1 ms in every CTA, the plan's status word reports
    it once, and the plan (and context) keep working (256: the line-pair
    kernel; 4096: its three-buffer ring variant)."""
    plan = _plan(N, I.random_symplectic_abcd(1), n, n)
    g = I.blob_field(n, n, seed=1)
    x = torch.from_numpy(g).to(torch.complex64).cuda()
    junk = torch.empty_like(x)
    assert N.nslct_status(plan.handle) == N.NSLCT_OK
    N.nslct_selftest_timeout(plan.handle, x, junk)
    torch.cuda.synchronize()
    assert N.nslct_status(plan.handle) == N.NSLCT_E_TIMEOUT
    assert N.nslct_status(plan.handle) == N.NSLCT_OK
    out = _gpu(plan, g)
    assert N.nslct_status(plan.handle) == N.NSLCT_OK
    assert O.rel_l2(out, _oracle(plan, g)) < TOL32


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fractional_fourier_eigenfunctions(N, precision):
    """The GPU chain keeps Hermite-Gaussians as eigenfunctions of the 2D
    fractional Fourier case (eigenvalue exp(-j (k + l + 1) phi))."""
    n, phi = 512, 0.7
    d = I.default_spacing(n)
    c, s = math.cos(phi), math.sin(phi)
    e = np.eye(2)
    m = np.block([[c * e, s * e], [-s * e, c * e]])
    plan = _plan(N, m, n, n, precision=precision)
    for k, l in [(0, 0), (2, 3), (6, 1)]:
        g = I.hg_field([(k, l)], n, d)
        out = _gpu(plan, g)
        lam = np.exp(-1j * (k + l + 1) * phi)
        assert O.rel_l2(out, lam * g) < (TOL32 if precision == "fp32" else 1e-11), (k, l)


def test_forward_group_equals_single_transforms(N):
    """nslct_forward_group runs independent transforms alternately on two
    streams: each output equals its single nslct_forward bit for bit, also for
    mixed sizes and schedules, in direct calls and on a side stream."""
    shapes = [(256, 256), (512, 128), (96, 64), (256, 256), (1024, 512)]
    plans, xs = [], []
    for k, (nx, ny) in enumerate(shapes):
        plans.append(_plan(N, I.random_symplectic_abcd(400 + k), nx, ny, method="lc_y" if k == 3 else "ha"))
        xs.append(torch.from_numpy(I.blob_field(nx, ny, seed=400 + k)).to(torch.complex64).cuda())
    outs = [torch.empty_like(x) for x in xs]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        N.nslct_forward_group([p.handle for p in plans], xs, outs, s)
    s.synchronize()
    for p, x, o in zip(plans, xs, outs):
        ref = p.forward(x)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)
