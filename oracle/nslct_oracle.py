"""FP64 CPU oracle for the 2D nonseparable discrete LCT (Pei & Huang,
"Two-dimensional nonseparable discrete linear canonical transform based on
CM-CC-CM-CC decomposition").

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports, calls or links
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may use it. It shares no code with the CUDA path.

What it computes, in the paper's own terms and order, as plain direct sums in
float64/complex128 (no FFT anywhere):

* ``cm``     -- 2D discrete chirp multiplication, Eq. BasicCM12 (Sec. 2.A).
* ``dft2`` / ``idft2`` -- 2D DFT / IDFT with the constant of Eqs. BasicDFT16/20
                (Sec. 2.B), evaluated as dense DFT-matrix products whose phases
                are reduced exactly as integers ((p*m) mod N) before ``exp``.
* ``cc``     -- 2D discrete chirp convolution F^-1 CM^{-B} F, Eq. BasicCC20 (Sec. 2.C).
* ``decompose`` -- the CM-CC-CM-CC factors of Eq. Bnonsym08 (Sec. 4.B):
                B' = B - AH, D' = D - CH, C2 = B'^-1 (A - I), C1 = (D' - I) B'^-1.
* ``forward`` -- the HA-NsDLCT chain of Eq. HA28, applied right to left:
                CC^H, then CM^{C2}, then CC^{B'}, then CM^{C1}.
* ``inverse`` -- the reversed chain with negated chirp matrices, Eq. CCCMCCCM04/30.
* ``ha_search`` -- a solver for the H criterion of Eq. HA24 (the paper names none).
* ``lc_h``    -- the closed-form one-parameter H of Eqs. LC04-LC10.
* ``direct``  -- the sampled continuous kernel ("direct method"), Eq. Intro32.
* ``project_sp4`` -- nearest-symplectic clean-up of 4-decimal printed matrices.

Readings taken where the paper is silent or ambiguous:

1. Index origin: samples are centred, m = i - floor(N/2) for storage index i;
   the same centred range is used for output and frequency indices.
2. F^-1 carries the constant (d_in_x * d_in_y) / (j 2 pi) built from ITS OWN
   input spacing (the frequency spacing 2 pi / (N dx)), so that CC^0 = -I and
   the chain is unitary (the paper states the matrix L of Eq. self12 is unitary).
3. All four operators are always executed, even when H = 0.
4. Output sampling equals input sampling (du = dx, dv = dy, Sec. 2.A).
5. Chirp matrices derived in floating point are symmetrised, c12 := (C12+C21)/2.
6. H search: lattice + shrinking-window refinement on the feasible plane
   (see ``ha_search``).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi

# --------------------------------------------------------------------------
# ABCD helpers (Eqs. Intro04, Intro12, Intro16)
# --------------------------------------------------------------------------


def split_abcd(m):
    """Return the 2x2 blocks A, B, C, D of a row-major 4x4 ABCD matrix (Eq. Intro04)."""
    m = np.asarray(m, dtype=np.float64).reshape(4, 4)
    return m[:2, :2].copy(), m[:2, 2:].copy(), m[2:, :2].copy(), m[2:, 2:].copy()


def symplectic_form():
    """J = (0, I; -I, 0)."""
    j = np.zeros((4, 4))
    j[:2, 2:] = np.eye(2)
    j[2:, :2] = -np.eye(2)
    return j


def symplectic_residual(m) -> float:
    """max |M^T J M - J|: zero exactly when the six constraints of Eq. Intro16 hold."""
    m = np.asarray(m, dtype=np.float64).reshape(4, 4)
    j = symplectic_form()
    return float(np.max(np.abs(m.T @ j @ m - j)))


def project_sp4(m, iters: int = 60):
    """Move a nearly symplectic matrix onto Sp(4).

    The paper prints its example matrices (Eqs. Acc24, Acc28, Add24, Add28) to
    four decimals, so they violate Eq. Intro12 by up to ~1e-3. The iteration
    X <- (X + J^T X^{-T} J) / 2 has every symplectic matrix as a fixed point
    (for symplectic X, J^T X^{-T} J = X) and converges quadratically from a
    nearby start.
    """
    x = np.asarray(m, dtype=np.float64).reshape(4, 4).copy()
    j = symplectic_form()
    for _ in range(iters):
        x_new = 0.5 * (x + j.T @ np.linalg.inv(x).T @ j)
        if np.max(np.abs(x_new - x)) < 1e-17:
            x = x_new
            break
        x = x_new
    return x


# --------------------------------------------------------------------------
# Basic discrete operators (Sec. 2)
# --------------------------------------------------------------------------


def centered(n: int) -> np.ndarray:
    """Centred integer indices m = i - floor(N/2), i = 0..N-1 (reading 1)."""
    return np.arange(n, dtype=np.int64) - n // 2


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """W[p, m] = exp(sign * j 2 pi (p m) / N) over centred p, m.

    The integer product p*m is reduced modulo N exactly before the exponential,
    so every entry is one of the N roots of unity computed from a small angle.
    """
    p = centered(n)
    e = np.mod(np.outer(p, p), n)
    return np.exp(sign * 1j * TWO_PI * e / n)


def cm(g: np.ndarray, c, du: float, dv: float) -> np.ndarray:
    """2D discrete chirp multiplication CM^C, Eq. BasicCM12 (Sec. 2.A).

    G[p,q] = exp(j/2 (c11 p^2 du^2 + 2 c12 p q du dv + c22 q^2 dv^2)) g[p,q]
    with centred p, q and the input's own sampling intervals du, dv.
    """
    c = np.asarray(c, dtype=np.float64)
    c11, c12, c22 = c[0, 0], 0.5 * (c[0, 1] + c[1, 0]), c[1, 1]
    nx, ny = g.shape
    p = centered(nx).astype(np.float64)[:, None] * du
    q = centered(ny).astype(np.float64)[None, :] * dv
    phase = 0.5 * (c11 * p * p + 2.0 * c12 * p * q + c22 * q * q)
    return np.exp(1j * phase) * g


def dft2(g: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """2D DFT F_{x,y} of Eq. BasicDFT16: (dx dy / (j 2 pi)) sum e^{-j2pi(pm+qn)/N} g[m,n]."""
    nx, ny = g.shape
    wx = dft_matrix(nx, -1)
    wy = dft_matrix(ny, -1)
    return (dx * dy / (1j * TWO_PI)) * (wx @ g @ wy.T)


def idft2(g: np.ndarray, du: float, dv: float) -> np.ndarray:
    """2D IDFT F^-1_{x,y} of Eq. BasicDFT20 with the constant (du dv)/(j 2 pi)
    built from its own input spacing du, dv (reading 2)."""
    nx, ny = g.shape
    wx = dft_matrix(nx, +1)
    wy = dft_matrix(ny, +1)
    return (du * dv / (1j * TWO_PI)) * (wx @ g @ wy.T)


def freq_spacing(n: int, d: float) -> float:
    """Output spacing of the DFT, du = 2 pi / (N dx) (Sec. 2.B)."""
    return TWO_PI / (n * d)


def cc(g: np.ndarray, b, dx: float, dy: float) -> np.ndarray:
    """2D discrete chirp convolution CC^B = F^-1 CM^{-B} F, Eq. BasicCC20 (Sec. 2.C).

    The chirp multiplication in the middle acts on the DFT output, whose
    sampling intervals are 2 pi / (N dx) and 2 pi / (N dy).
    """
    nx, ny = g.shape
    dwx, dwy = freq_spacing(nx, dx), freq_spacing(ny, dy)
    spec = dft2(g, dx, dy)
    spec = cm(spec, -np.asarray(b, dtype=np.float64), dwx, dwy)
    return idft2(spec, dwx, dwy)


# --------------------------------------------------------------------------
# CM-CC-CM-CC decomposition (Sec. 4.B)
# --------------------------------------------------------------------------


def sym_part(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * (x + x.T)


def decompose(m, h):
    """Factors of Eq. Bnonsym08 for a symmetric H.

    Returns dict with H, Bp (= B - AH, Eq. Bnonsym04), Dp (= D - CH),
    C2 (= Bp^-1 (A - I), the CM applied second) and C1 (= (Dp - I) Bp^-1, the
    CM applied last). C1 and C2 are symmetric in exact arithmetic when Bp is
    (reading 5 symmetrises them).
    """
    a, b, c, d = split_abcd(m)
    h = sym_part(h)
    eye = np.eye(2)
    bp = b - a @ h
    dp = d - c @ h
    bpi = np.linalg.inv(bp)
    c2 = bpi @ (a - eye)
    c1 = (dp - eye) @ bpi
    return {"H": h, "Bp": sym_part(bp), "Dp": dp, "C1": sym_part(c1), "C2": sym_part(c2),
            "Bp_asym": float(abs(bp[0, 1] - bp[1, 0])),
            "C_asym": float(max(abs(c1[0, 1] - c1[1, 0]), abs(c2[0, 1] - c2[1, 0])))}


def compose_factors(params):
    """Product (I,0;C1,I)(I,Bp;0,I)(I,0;C2,I)(I,H;0,I) of Eq. Bnonsym08."""
    eye = np.eye(2)
    zero = np.zeros((2, 2))

    def cmm(c):
        return np.block([[eye, zero], [c, eye]])

    def ccm(b):
        return np.block([[eye, b], [zero, eye]])

    return cmm(params["C1"]) @ ccm(params["Bp"]) @ cmm(params["C2"]) @ ccm(params["H"])


def gamma(c) -> float:
    """Space-bandwidth growth ratio of Eq. HA16 for a symmetric 2x2 matrix."""
    c = np.asarray(c, dtype=np.float64)
    c11, c12, c22 = abs(c[0, 0]), abs(0.5 * (c[0, 1] + c[1, 0])), abs(c[1, 1])
    return (c11 + c12 + 1.0) * (c12 + c22 + 1.0)


def ha_objective(m, h) -> float:
    """Objective of Eq. HA24: gamma(C1) gamma(B') gamma(C2) gamma(H)."""
    p = decompose(m, h)
    return gamma(p["C1"]) * gamma(p["Bp"]) * gamma(p["C2"]) * gamma(p["H"])


def feasible_plane(m):
    """Linear condition on h = (h11, h12, h22) for B - AH to be symmetric
    (the requirement B' = B'^T of Eq. Bnonsym32).

    (B - AH)_12 = (B - AH)_21 gives  r . h = rhs  with
    r = (-a21, a11 - a22, a12), rhs = b12 - b21.  Setting h12 = h22 = 0 or
    h11 = h12 = 0 recovers Eqs. LC08 and LC10.
    """
    a, b, _, _ = split_abcd(m)
    r = np.array([-a[1, 0], a[0, 0] - a[1, 1], a[0, 1]])
    rhs = b[0, 1] - b[1, 0]
    return r, rhs


def h_from_vec(v):
    return np.array([[v[0], v[1]], [v[1], v[2]]], dtype=np.float64)


DET_FLOOR = 1e-3


def _objective_vec(m, hv):
    h = h_from_vec(hv)
    a, b, c, d = split_abcd(m)
    bp = b - a @ h
    det = bp[0, 0] * bp[1, 1] - bp[0, 1] * bp[1, 0]
    if not np.isfinite(det) or abs(det) < DET_FLOOR:
        return math.inf
    return ha_objective(m, h)


def _grid_objective(m, hs):
    """Vectorised Eq. HA24 objective for an array of h vectors (K, 3)."""
    a, b, c, d = split_abcd(m)
    h11, h12, h22 = hs[:, 0], hs[:, 1], hs[:, 2]
    # B' = B - A H
    bp11 = b[0, 0] - (a[0, 0] * h11 + a[0, 1] * h12)
    bp12 = b[0, 1] - (a[0, 0] * h12 + a[0, 1] * h22)
    bp21 = b[1, 0] - (a[1, 0] * h11 + a[1, 1] * h12)
    bp22 = b[1, 1] - (a[1, 0] * h12 + a[1, 1] * h22)
    # D' = D - C H
    dp11 = d[0, 0] - (c[0, 0] * h11 + c[0, 1] * h12)
    dp12 = d[0, 1] - (c[0, 0] * h12 + c[0, 1] * h22)
    dp21 = d[1, 0] - (c[1, 0] * h11 + c[1, 1] * h12)
    dp22 = d[1, 1] - (c[1, 0] * h12 + c[1, 1] * h22)
    det = bp11 * bp22 - bp12 * bp21
    ok = np.abs(det) >= DET_FLOOR
    det = np.where(ok, det, 1.0)
    i11, i12, i21, i22 = bp22 / det, -bp12 / det, -bp21 / det, bp11 / det
    # C2 = B'^-1 (A - I)
    am = a - np.eye(2)
    c2_11 = i11 * am[0, 0] + i12 * am[1, 0]
    c2_12 = i11 * am[0, 1] + i12 * am[1, 1]
    c2_21 = i21 * am[0, 0] + i22 * am[1, 0]
    c2_22 = i21 * am[0, 1] + i22 * am[1, 1]
    # C1 = (D' - I) B'^-1
    e11, e12, e21, e22 = dp11 - 1.0, dp12, dp21, dp22 - 1.0
    c1_11 = e11 * i11 + e12 * i21
    c1_12 = e11 * i12 + e12 * i22
    c1_21 = e21 * i11 + e22 * i21
    c1_22 = e21 * i12 + e22 * i22

    def g(x11, x12, x21, x22):
        s = np.abs(0.5 * (x12 + x21))
        return (np.abs(x11) + s + 1.0) * (s + np.abs(x22) + 1.0)

    obj = g(c1_11, c1_12, c1_21, c1_22) * g(bp11, bp12, bp21, bp22) * \
        g(c2_11, c2_12, c2_21, c2_22) * g(h11, h12, h12, h22)
    return np.where(ok, obj, np.inf)


def ha_search(m, grid: int = 241, grid3: int = 41, starts: int = 6, zoom_pts: int = 21,
              tol: float = 1e-11):
    """Choose H by the high-accuracy criterion of Eq. HA24 (Sec. 4.B.1).

    The paper gives the criterion, not a solver. This one:
    1. restricts h = (h11, h12, h22) to the feasible plane r.h = rhs
       (``feasible_plane``), parametrised h = h0 + s e1 + t e2 with h0 the
       minimum-norm point and (e1, e2) an orthonormal basis of the plane's
       direction space;
    2. scans a ``grid`` x ``grid`` lattice over s, t in [-R, R],
       R = 6 max(1, max|M|), discarding points with |det B'| < 1e-3;
    3. refines each of the ``starts`` best lattice points (taken at least two
       lattice steps apart) by a shrinking-window search: a ``zoom_pts`` x
       ``zoom_pts`` grid around the current point, re-centred on its best
       entry, with the window quartered each round until it is below ``tol``.
       A full window (not a compass) is used because the objective has kinks
       (absolute values in Eq. HA16) along which axis moves stall.
    If r = 0 the plane degenerates: with rhs = 0 every symmetric H is feasible
    and the same is done in three dimensions (``grid3`` lattice, 9^3 windows);
    otherwise no symmetric H exists and ValueError is raised.
    Returns the symmetric 2x2 H with the lowest objective found.
    """
    m = np.asarray(m, dtype=np.float64).reshape(4, 4)
    r, rhs = feasible_plane(m)
    rn = float(np.linalg.norm(r))
    scale = 6.0 * max(1.0, float(np.max(np.abs(m))))
    if rn > 1e-12:
        h0 = r * (rhs / (rn * rn))
        _, _, vt = np.linalg.svd(r.reshape(1, 3))
        basis = vt[1:3]  # orthonormal rows orthogonal to r
        dim = 2
        lat = np.linspace(-scale, scale, grid)
        coords = np.stack(np.meshgrid(lat, lat, indexing="ij"), axis=-1).reshape(-1, 2)

        def points(c):
            return h0[None, :] + c[:, 0:1] * basis[0][None, :] + c[:, 1:2] * basis[1][None, :]
        step0 = lat[1] - lat[0]
        wpts = zoom_pts
    else:
        if abs(rhs) > 1e-12:
            raise ValueError("ha_search: B - AH cannot be symmetric for any symmetric H")
        dim = 3
        lat = np.linspace(-scale, scale, grid3)
        coords = np.stack(np.meshgrid(lat, lat, lat, indexing="ij"), axis=-1).reshape(-1, 3)

        def points(c):
            return c
        step0 = lat[1] - lat[0]
        wpts = 9
    obj = _grid_objective(m, points(coords))
    order = np.argsort(obj, kind="stable")
    if not np.isfinite(obj[order[0]]):
        raise ValueError("ha_search: no feasible H with |det B'| >= floor on the lattice")
    seeds = []
    for k in order:
        if not np.isfinite(obj[k]) or len(seeds) >= starts:
            break
        c = coords[k]
        if all(np.max(np.abs(c - s0)) > 2.5 * step0 for s0 in seeds):
            seeds.append(c.copy())
    offs1 = np.linspace(-1.0, 1.0, wpts)
    offs = np.stack(np.meshgrid(*([offs1] * dim), indexing="ij"), axis=-1).reshape(-1, dim)
    best_c, best_v = None, math.inf
    for c in seeds:
        cur = c.copy()
        cur_v = float(_grid_objective(m, points(cur[None, :]))[0])
        half = step0
        while half > tol:
            cand = cur[None, :] + half * offs
            vals = _grid_objective(m, points(cand))
            k = int(np.argmin(vals))
            if vals[k] < cur_v:
                cur, cur_v = cand[k].copy(), float(vals[k])
            half *= 0.25
        if cur_v < best_v:
            best_c, best_v = cur, cur_v
    return h_from_vec(points(best_c[None, :])[0])


def lc_h(m, only_y: bool = False):
    """Low-complexity H of Eqs. LC04-LC10 (Sec. 4.B.2).

    Candidates: H = (h,0;0,0) with h = (b21 - b12)/a21 when a21 != 0, and
    H = (0,0;0,h) with h = (b12 - b21)/a12 when a12 != 0. Candidates whose B'
    is (numerically) singular are dropped; of the rest the one with the lower
    Eq. HA24 objective is returned. Returns None when no candidate is valid
    (the paper then falls back to the HA choice). ``only_y`` keeps the
    Eq. LC10 candidate alone.
    """
    a, b, _, _ = split_abcd(m)
    cands = []
    if abs(a[1, 0]) > 1e-12 and not only_y:
        cands.append(np.array([[(b[1, 0] - b[0, 1]) / a[1, 0], 0.0], [0.0, 0.0]]))
    if abs(a[0, 1]) > 1e-12:
        cands.append(np.array([[0.0, 0.0], [0.0, (b[0, 1] - b[1, 0]) / a[0, 1]]]))
    best, best_obj = None, math.inf
    for h in cands:
        bp = b - a @ h
        if abs(np.linalg.det(bp)) < DET_FLOOR:
            continue
        val = ha_objective(m, h)
        if val < best_obj:
            best, best_obj = h, val
    return best


def plan(m, h=None, method: str = "ha"):
    """Decomposition parameters for ABCD ``m``: H from ``h`` if given, else by
    the HA search (Eq. HA24) or the LC closed form (Eqs. LC08/LC10)."""
    m = np.asarray(m, dtype=np.float64).reshape(4, 4)
    if h is None:
        if method == "lc":
            h = lc_h(m)
            if h is None:
                h = ha_search(m)
        else:
            h = ha_search(m)
    return decompose(m, h)


# --------------------------------------------------------------------------
# The NsDLCT chain (Sec. 4.B, Eq. HA28) and its exact inverse (Sec. 4.C)
# --------------------------------------------------------------------------


def forward(g, params, dx: float, dy: float) -> np.ndarray:
    """HA-NsDLCT of Eq. HA28, applied right to left:
    CC^H, then CM^{C2} with C2 = B'^-1(A - I), then CC^{B'}, then CM^{C1}
    with C1 = (D' - I) B'^-1. Output spacing equals input spacing."""
    x = np.asarray(g, dtype=np.complex128)
    x = cc(x, params["H"], dx, dy)
    x = cm(x, params["C2"], dx, dy)
    x = cc(x, params["Bp"], dx, dy)
    x = cm(x, params["C1"], dx, dy)
    return x


def inverse(big_g, params, dx: float, dy: float) -> np.ndarray:
    """Inverse chain of Eq. CCCMCCCM04 (= Eq. CCCMCCCM30), applied right to left:
    CM^{-C1}, then CC^{-B'}, then CM^{-C2}, then CC^{-H}."""
    x = np.asarray(big_g, dtype=np.complex128)
    x = cm(x, -params["C1"], dx, dy)
    x = cc(x, -params["Bp"], dx, dy)
    x = cm(x, -params["C2"], dx, dy)
    x = cc(x, -params["H"], dx, dy)
    return x


# --------------------------------------------------------------------------
# CC-CM-CC-CM ("type 2") decomposition (Sec. 4.C) and the tr(B) rule of
# Eq. Reversible08
# --------------------------------------------------------------------------


def decompose_type2(m, h1):
    """Factors of Eq. CCCMCCCM16 for a symmetric H1:
    B1' = B - H1 D and A1' = A - H1 C (Eq. CCCMCCCM23 before substitution),
    Ca = B1'^-1 (A1' - I) (the CM applied first) and Cb = (D - I) B1'^-1 (the
    CM applied third); the chain is CM^{Ca}, CC^{B1'}, CM^{Cb}, CC^{H1}.
    B1' must be symmetric (the CC's chirp matrix), which constrains H1."""
    a, b, c, d = split_abcd(m)
    h1 = sym_part(h1)
    eye = np.eye(2)
    bp1 = b - h1 @ d
    ap1 = a - h1 @ c
    bpi = np.linalg.inv(bp1)
    ca = bpi @ (ap1 - eye)
    cb = (d - eye) @ bpi
    return {"H1": h1, "Bp1": sym_part(bp1), "Ap1": ap1, "Ca": sym_part(ca), "Cb": sym_part(cb),
            "Bp1_asym": float(abs(bp1[0, 1] - bp1[1, 0]))}


def compose_factors_type2(p2):
    """(I, H1; 0, I)(I, 0; Cb, I)(I, B1'; 0, I)(I, 0; Ca, I): the ABCD matrix
    the type-2 chain stands for (CC^B <-> (I, B; 0, I), CM^C <-> (I, 0; C, I))."""
    eye, z = np.eye(2), np.zeros((2, 2))
    cc_m = lambda bb: np.block([[eye, bb], [z, eye]])
    cm_m = lambda cc_: np.block([[eye, z], [cc_, eye]])
    return cc_m(p2["H1"]) @ cm_m(p2["Cb"]) @ cc_m(p2["Bp1"]) @ cm_m(p2["Ca"])


def ha_objective_type2(m, h1) -> float:
    """The HA criterion carried to the type-2 chain: the product of the four
    chirps' gamma factors, gamma(Ca) gamma(B1') gamma(Cb) gamma(H1)."""
    p = decompose_type2(m, h1)
    return gamma(p["Ca"]) * gamma(p["Bp1"]) * gamma(p["Cb"]) * gamma(p["H1"])


def symplectic_inverse(m):
    """(A, B; C, D)^-1 = (D^T, -B^T; -C^T, A^T) (Eq. CCCMCCCM20)."""
    a, b, c, d = split_abcd(m)
    return np.block([[d.T, -b.T], [-c.T, a.T]])


def plan_type2(m, h1=None, method: str = "ha"):
    """Type-2 factors for ABCD ``m``. H1 minimises the type-2 HA criterion;
    since B1'(M, H1) = -B'(M^-1, -H1)^T (Eq. CCCMCCCM24) and likewise for the
    other three chirps, and gamma depends on absolute values of a symmetric
    matrix only, that criterion equals the type-1 one of M^-1 at -H1, so the
    type-1 search on M^-1 is reused: H1 = -H(M^-1). ``method="lc"`` takes the
    closed forms of Eqs. LC08/LC10 the same way."""
    m = np.asarray(m, dtype=np.float64).reshape(4, 4)
    if h1 is None:
        mi = symplectic_inverse(m)
        if method == "lc":
            h = lc_h(mi)
            if h is None:
                h = ha_search(mi)
        else:
            h = ha_search(mi)
        h1 = -h
    return decompose_type2(m, h1)


def forward_type2(g, p2, dx: float, dy: float) -> np.ndarray:
    """Eq. CCCMCCCM16 applied right to left: CM^{Ca}, CC^{B1'}, CM^{Cb}, CC^{H1}."""
    x = np.asarray(g, dtype=np.complex128)
    x = cm(x, p2["Ca"], dx, dy)
    x = cc(x, p2["Bp1"], dx, dy)
    x = cm(x, p2["Cb"], dx, dy)
    x = cc(x, p2["H1"], dx, dy)
    return x


def inverse_type2(big_g, p2, dx: float, dy: float) -> np.ndarray:
    """The type-2 chain reversed with every chirp negated (its exact inverse)."""
    x = np.asarray(big_g, dtype=np.complex128)
    x = cc(x, -p2["H1"], dx, dy)
    x = cm(x, -p2["Cb"], dx, dy)
    x = cc(x, -p2["Bp1"], dx, dy)
    x = cm(x, -p2["Ca"], dx, dy)
    return x


def uses_type2(m) -> bool:
    """Eq. Reversible08: type 1 for tr(B) > 0, type 2 for tr(B) < 0; tr(B) = 0,
    which the equation leaves open, is taken as type 1."""
    _, b, _, _ = split_abcd(m)
    return float(np.trace(b)) < 0.0


def zero_pad(g, nx_pad: int, ny_pad: int) -> np.ndarray:
    """Zero-pad an Nx x Ny field to Nx_pad x Ny_pad (Sec. 2.A; Sec. 5.A pads
    the input to (N + dN) x (N + dN) against aliasing) keeping each sample at
    its centred index: row i of the field (index i - floor(Nx/2)) becomes row
    i + floor(Nx_pad/2) - floor(Nx/2) of the padded grid."""
    g = np.asarray(g, dtype=np.complex128)
    nx, ny = g.shape
    out = np.zeros((nx_pad, ny_pad), dtype=np.complex128)
    r0, c0 = nx_pad // 2 - nx // 2, ny_pad // 2 - ny // 2
    out[r0:r0 + nx, c0:c0 + ny] = g
    return out


def centre_crop(x, nx: int, ny: int) -> np.ndarray:
    """The Nx x Ny region of a larger grid at the same centred indices (the
    inverse of zero_pad on its support)."""
    x = np.asarray(x)
    r0, c0 = x.shape[0] // 2 - nx // 2, x.shape[1] // 2 - ny // 2
    return x[r0:r0 + nx, c0:c0 + ny]


def forward_padded(g, params, dx: float, dy: float, nx_pad: int, ny_pad: int, crop: bool = False):
    """The chain of Eq. HA28 on the zero-padded input, with the same sample
    spacing (so the frequency spacing becomes 2 pi / (N_pad dx)); the whole
    padded output, or its centred input-sized region."""
    out = forward(zero_pad(g, nx_pad, ny_pad), params, dx, dy)
    return centre_crop(out, *np.shape(g)) if crop else out


def inverse_padded(big_g, params, dx: float, dy: float, nx_pad: int, ny_pad: int, nx: int, ny: int):
    """Inverse chain on the padded grid: the input (the padded output, or its
    centred crop) is zero-padded to the grid, and the centred Nx x Ny region
    of the result is returned."""
    return centre_crop(inverse(zero_pad(big_g, nx_pad, ny_pad), params, dx, dy), nx, ny)


def filter_two_domains(g, params1, params3, h1, h3, dx: float, dy: float):
    """Eq. Add04: filter h1 in the NsLCT domain of M1, then h3 in that of M3,
    and back to space through both inverses (each the exact inverse chain of
    its plan, Eq. CCCMCCCM04). The (A3,B3;C3,D2) printed inside Eq. Add04 is
    read as M3."""
    y = np.asarray(h1) * forward(g, params1, dx, dy)
    y = np.asarray(h3) * forward(y, params3, dx, dy)
    return inverse(inverse(y, params3, dx, dy), params1, dx, dy)


def filter_two_domains_additive(g, params1, params3, params31, h1, h3, dx: float, dy: float):
    """Eq. Add08: the same two filters, but one inverse transform of the
    composed matrix M3 M1 (params31) replaces the two inverses; exact only
    if the NsDLCT were additive."""
    y = np.asarray(h1) * forward(g, params1, dx, dy)
    y = np.asarray(h3) * forward(y, params3, dx, dy)
    return inverse(y, params31, dx, dy)


def nmse_add(g, params1, params3, params31, dx: float, dy: float) -> float:
    """Eq. Add16 with G = L_{M3}(L_{M1} g) (Eq. Add20) and G' = L_{M3 M1} g (Eq. Add22)."""
    big = forward(forward(g, params1, dx, dy), params3, dx, dy)
    return nmse(forward(g, params31, dx, dy), big)


def transform(g, m, dx: float, dy: float, h=None, method: str = "ha"):
    """Plan and apply the NsDLCT for ABCD ``m``."""
    return forward(g, plan(m, h=h, method=method), dx, dy)


# --------------------------------------------------------------------------
# Direct method (Eq. Intro32) and error measures (Sec. 5)
# --------------------------------------------------------------------------


def direct(g, m, dx: float, dy: float, du: float, dv: float, nout_x: int, nout_y: int):
    """Direct method of Eq. Intro32: the continuous kernel of Eq. Intro08
    sampled at input points r = (m dx, n dy) and output points r' = (p du, q dv)
    (all centred), summed with weight dx dy.

    The cross term -2 r^T B^-1 r' is split per output row p, which turns the
    O(N^4) sum into one matrix product per p; nothing is approximated.
    The square root sqrt(-det B) is the principal complex root.
    """
    a, b, c, d = split_abcd(m)
    bi = np.linalg.inv(b)
    bia = bi @ a
    dbi = d @ bi
    nx, ny = g.shape
    x = centered(nx) * dx
    y = centered(ny) * dy
    u = centered(nout_x) * du
    v = centered(nout_y) * dv
    xx, yy = x[:, None], y[None, :]
    qin = np.exp(0.5j * (xx * bia[0, 0] * xx + xx * bia[0, 1] * yy + yy * bia[1, 0] * xx + yy * bia[1, 1] * yy))
    uu, vv = u[:, None], v[None, :]
    qout = np.exp(0.5j * (uu * dbi[0, 0] * uu + uu * dbi[0, 1] * vv + vv * dbi[1, 0] * uu + vv * dbi[1, 1] * vv))
    h = qin * np.asarray(g, dtype=np.complex128)
    # exp(-j r^T B^-1 r') = exp(-j (x bi11 u + x bi12 v + y bi21 u + y bi22 v))
    vmat = np.exp(-1j * np.outer(v, y) * bi[1, 1])  # [q, n]
    umat = np.exp(-1j * np.outer(v, x) * bi[0, 1])  # [q, m]
    out = np.empty((nout_x, nout_y), dtype=np.complex128)
    for ip, up in enumerate(u):
        hp = h * np.exp(-1j * x * bi[0, 0] * up)[:, None] * np.exp(-1j * y * bi[1, 0] * up)[None, :]
        z = hp @ vmat.T  # [m, q]
        out[ip] = np.sum(umat * z.T, axis=1)
    pref = dx * dy / (TWO_PI * np.sqrt(complex(-np.linalg.det(b))))
    return pref * qout * out


def nmse(approx, ref) -> float:
    """Normalised mean-square error of Eqs. Acc04, Add16, Rev08."""
    approx = np.asarray(approx)
    ref = np.asarray(ref)
    return float(np.sum(np.abs(approx - ref) ** 2) / np.sum(np.abs(ref) ** 2))


def rel_l2(approx, ref) -> float:
    """Relative L2 error ||approx - ref|| / ||ref||."""
    return math.sqrt(nmse(approx, ref))


# --------------------------------------------------------------------------
# Gradients of a real loss through the chain (adjoint of Eq. HA28)
# --------------------------------------------------------------------------
#
# Parameters. An ABCD matrix with invertible A is written as
#   M(theta) = (I, 0; C, I) (L, 0; 0, L^-T) (I, B; 0, I) = (L, L B; C L, C L B + L^-T)
# with C, B symmetric (3 + 3 entries) and L = A (4 entries): the 10 degrees of
# freedom of Sec. 1 (Eq. Intro12 leaves 10 of 16). theta = (c11, c12, c22,
# l11, l12, l21, l22, b11, b12, b22).
# H(theta): a reference H0 moved onto the feasible plane of M(theta) along the
# plane's normal, H0 + r (rhs - r.h0) / |r|^2 (smooth in theta; equals H0 when
# H0 is feasible).


def theta_from_abcd(m):
    """theta of M: L = A, C = sym(C A^-1), B = sym(A^-1 B)."""
    a, b, c, _ = split_abcd(m)
    ai = np.linalg.inv(a)
    cs = sym_part(c @ ai)
    bs = sym_part(ai @ b)
    return np.array([cs[0, 0], cs[0, 1], cs[1, 1], a[0, 0], a[0, 1], a[1, 0], a[1, 1],
                     bs[0, 0], bs[0, 1], bs[1, 1]])


def abcd_from_theta(th):
    """(I,0;C,I)(L,0;0,L^-T)(I,B;0,I) for theta (works for complex theta)."""
    th = np.asarray(th)
    dt = np.result_type(th.dtype, np.float64)
    c = np.array([[th[0], th[1]], [th[1], th[2]]], dtype=dt)
    lm = np.array([[th[3], th[4]], [th[5], th[6]]], dtype=dt)
    b = np.array([[th[7], th[8]], [th[8], th[9]]], dtype=dt)
    eye = np.eye(2, dtype=dt)
    z = np.zeros((2, 2), dtype=dt)
    lit = np.linalg.inv(lm).T
    return np.block([[eye, z], [c, eye]]) @ np.block([[lm, z], [z, lit]]) @ np.block([[eye, b], [z, eye]])


def h_of_theta(th, h0):
    """H0 moved along the normal r onto the feasible plane r.h = rhs of M(theta)."""
    m = abcd_from_theta(th)
    a, b = m[:2, :2], m[:2, 2:]
    r = np.array([-a[1, 0], a[0, 0] - a[1, 1], a[0, 1]])
    rhs = b[0, 1] - b[1, 0]
    hv = np.array([h0[0, 0], 0.5 * (h0[0, 1] + h0[1, 0]), h0[1, 1]], dtype=r.dtype)
    rr = r @ r  # no conjugate: analytic in theta (complex-step friendly)
    if abs(rr) < 1e-24:
        v = hv
    else:
        v = hv + r * (rhs - r @ hv) / rr
    return np.array([[v[0], v[1]], [v[1], v[2]]])


def _chirp_vec(th, h0):
    """(H, B', C1, C2) symmetric entries (12 values) as functions of theta, in
    the order h11 h12 h22, b'11 b'12 b'22, c1_11 c1_12 c1_22, c2_11 c2_12 c2_22."""
    m = abcd_from_theta(th)
    h = h_of_theta(th, h0)
    a, b, c, d = m[:2, :2], m[:2, 2:], m[2:, :2], m[2:, 2:]
    eye = np.eye(2)
    bp = b - a @ h
    dp = d - c @ h
    bpi = np.linalg.inv(bp)
    c2 = bpi @ (a - eye)
    c1 = (dp - eye) @ bpi
    out = []
    for x in (h, bp, c1, c2):
        out += [x[0, 0], 0.5 * (x[0, 1] + x[1, 0]), x[1, 1]]
    return np.array(out)


def chirp_jacobian(th, h0, step: float = 1e-30):
    """d(chirp entries)/d(theta), 12 x 10, by the complex-step derivative
    Im f(theta + i s e_k) / s: every operation in _chirp_vec is analytic, so the
    result is exact to rounding (no subtraction error)."""
    th = np.asarray(th, dtype=np.float64)
    jac = np.zeros((12, 10))
    for k in range(10):
        tc = th.astype(np.complex128)
        tc[k] += 1j * step
        jac[:, k] = np.imag(_chirp_vec(tc, h0)) / step
    return jac


def params_from_theta(th, h0):
    m = abcd_from_theta(np.asarray(th, dtype=np.float64))
    return decompose(m, h_of_theta(np.asarray(th, dtype=np.float64), h0))


def dft2_adj(g, dx, dy):
    """Adjoint of dft2: conj(constant) * W^H g conj(W)^... (W symmetric)."""
    nx, ny = g.shape
    wx = dft_matrix(nx, +1)
    wy = dft_matrix(ny, +1)
    return np.conj(dx * dy / (1j * TWO_PI)) * (wx @ g @ wy.T)


def idft2_adj(g, du, dv):
    nx, ny = g.shape
    wx = dft_matrix(nx, -1)
    wy = dft_matrix(ny, -1)
    return np.conj(du * dv / (1j * TWO_PI)) * (wx @ g @ wy.T)


def _phase_weights(nx, ny, du, dv, sign):
    """d phi / d(c11, c12, c22) of a chirp exp(j sign/2 (c11 p^2 du^2 + 2 c12 p q du dv + c22 q^2 dv^2))."""
    p = centered(nx).astype(np.float64)[:, None] * du
    q = centered(ny).astype(np.float64)[None, :] * dv
    return (sign * 0.5 * p * p * np.ones((1, ny)), sign * p * q, sign * 0.5 * q * q * np.ones((nx, 1)))


def chain_vjp(x, gbar, params, dx, dy, with_abs: bool = False):
    """Gradient of a real loss l(y), y = forward(x), given gbar = dl/dRe y + j dl/dIm y.

    Returns (grad_x, grad_chirp[, abs_chirp]) where grad_x = L^H gbar and grad_chirp holds
    dl/d(h11, h12, h22, b'11, b'12, b'22, c1_11, c1_12, c1_22, c2_11, c2_12, c2_22)
    (symmetric off-diagonal entries counted once, as they enter the phases).
    Every chirp stage v_out = e^{j phi(c)} v_in contributes
    dl/dc = Re sum conj(gbar_s) j (dphi/dc) v_out = -sum (dphi/dc) Im(conj(gbar_s) v_out),
    where gbar_s is gbar pulled back through the later stages by their adjoints.
    With ``with_abs`` also returns sum |dphi/dc| |gbar_s| |v_out| per entry: the
    scale against which rounding in the fields (not in this sum) is measured.
    """
    nx, ny = x.shape
    dwx, dwy = freq_spacing(nx, dx), freq_spacing(ny, dy)
    x = np.asarray(x, dtype=np.complex128)
    # forward, keeping each chirp stage's output (application order of Eq. HA28)
    f0 = dft2(x, dx, dy)
    v1 = cm(f0, -params["H"], dwx, dwy)
    w1 = idft2(v1, dwx, dwy)
    v2 = cm(w1, params["C2"], dx, dy)
    f2 = dft2(v2, dx, dy)
    v3 = cm(f2, -params["Bp"], dwx, dwy)
    w3 = idft2(v3, dwx, dwy)
    v4 = cm(w3, params["C1"], dx, dy)
    # backward
    g4 = np.asarray(gbar, dtype=np.complex128)
    g3 = idft2_adj(cm(g4, -params["C1"], dx, dy), dwx, dwy)
    g2 = dft2_adj(cm(g3, params["Bp"], dwx, dwy), dx, dy)
    g1 = idft2_adj(cm(g2, -params["C2"], dx, dy), dwx, dwy)
    gx = dft2_adj(cm(g1, params["H"], dwx, dwy), dx, dy)

    def contrib(g, v, weights):
        q = np.imag(np.conj(g) * v)
        return [-float(np.sum(w * q)) for w in weights]

    def magnitude(g, v, weights):
        q = np.abs(g) * np.abs(v)
        return [float(np.sum(np.abs(w) * q)) for w in weights]

    stages = [(g1, v1, _phase_weights(nx, ny, dwx, dwy, -1.0)),   # H (CM^{-H} in frequency)
              (g3, v3, _phase_weights(nx, ny, dwx, dwy, -1.0)),   # B'
              (g4, v4, _phase_weights(nx, ny, dx, dy, +1.0)),     # C1
              (g2, v2, _phase_weights(nx, ny, dx, dy, +1.0))]     # C2
    grad = []
    for g, v, w in stages:
        grad += contrib(g, v, w)
    if with_abs:
        mag = []
        for g, v, w in stages:
            mag += magnitude(g, v, w)
        return gx, np.array(grad), np.array(mag)
    return gx, np.array(grad)


def loss_and_grad(x, y_target, m, h0, dx, dy):
    """l = ||forward(x; theta) - y_target||^2 with theta = theta_from_abcd(m) and
    H = h_of_theta(theta, h0). Returns (l, dl/dRe x + j dl/dIm x, dl/dtheta[10],
    dl/dchirp[12])."""
    th = theta_from_abcd(m)
    params = params_from_theta(th, h0)
    y = forward(x, params, dx, dy)
    r = y - y_target
    loss = float(np.sum(np.abs(r) ** 2))
    gx, gch = chain_vjp(x, 2.0 * r, params, dx, dy)
    gth = chirp_jacobian(th, h0).T @ gch
    return loss, gx, gth, gch
