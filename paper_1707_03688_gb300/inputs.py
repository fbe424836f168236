"""Seeded synthetic inputs for the 2D NsDLCT (fields and ABCD matrices).

This module holds input generation only: no step of the transform itself lives
here. It is the one module that both the CUDA path's tests/bench and the FP64
oracle's tests draw their inputs from, so that both sides see identical data.

Generators
----------
* ``blob_field``      -- sum of complex Gaussian blobs (the synthetic stand-in for
                         the paper's smooth test images, Sec. 5 / Fig. 1).
* ``add_white_noise`` -- circular complex white noise of a given sigma.
* ``hermite_gaussian_1d`` / ``hg_field`` -- the paper's Hermite-Gaussian test
                         signals (Sec. 5.A, Eqs. Acc12-Acc20).
* ``random_symplectic_abcd`` -- random real 4x4 symplectic matrices built as
                         lower shear x rotation-gyrator x upper shear (the constraints of
                         Eq. Intro12 hold by construction).
* ``default_spacing`` -- the paper's sampling condition dx*du = 2*pi/N with
                         du = dx (Sec. 2.B), i.e. dx = sqrt(2*pi/N).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "blob_field",
    "add_white_noise",
    "gaussian_mask",
    "hermite_gaussian_1d",
    "hg_field",
    "random_symplectic_abcd",
    "default_spacing",
    "centered_coords",
]


def default_spacing(n: int) -> float:
    """Sampling interval satisfying dx^2 = 2*pi/N (Sec. 2.B, condition of Eq. BasicDFT16)."""
    return math.sqrt(2.0 * math.pi / n)


def centered_coords(n: int) -> np.ndarray:
    """Integer sample indices m = i - floor(N/2), i = 0..N-1 (the centred grid)."""
    return np.arange(n, dtype=np.int64) - n // 2


def blob_field(nx: int, ny: int, seed: int, nblobs: int = 8,
               width_range=(2.0, 8.0), dtype=np.complex128) -> np.ndarray:
    """Sum of ``nblobs`` complex Gaussian blobs on an nx x ny grid.

    Each blob has unit amplitude, a phase U(0, 2pi), a centre uniform over the
    grid and a width U(width_range) in pixels:
    ``exp(j psi) * exp(-|r - c|^2 / (2 w^2))``. Row index i runs along x.
    """
    rng = np.random.default_rng(seed)
    i = np.arange(nx, dtype=np.float64)[:, None]
    j = np.arange(ny, dtype=np.float64)[None, :]
    out = np.zeros((nx, ny), dtype=np.complex128)
    for _ in range(nblobs):
        ci = rng.uniform(0, nx)
        cj = rng.uniform(0, ny)
        w = rng.uniform(*width_range)
        psi = rng.uniform(0, 2 * math.pi)
        # separable evaluation keeps large grids cheap
        ex = np.exp(-((i - ci) ** 2) / (2 * w * w))
        ey = np.exp(-((j - cj) ** 2) / (2 * w * w))
        out += (math.cos(psi) + 1j * math.sin(psi)) * (ex * ey)
    return out.astype(dtype)


def gaussian_mask(nx: int, ny: int, sigma_frac: float = 0.25, tilt: float = 0.0,
                  dtype=np.complex128) -> np.ndarray:
    """A smooth filter for the NsLCT domain: a centred Gaussian window of
    width sigma_frac * N (in samples) times a linear phase exp(j tilt p / N),
    with p the centred row index."""
    p = (np.arange(nx) - nx // 2)[:, None].astype(np.float64)
    q = (np.arange(ny) - ny // 2)[None, :].astype(np.float64)
    w = np.exp(-0.5 * ((p / (sigma_frac * nx)) ** 2 + (q / (sigma_frac * ny)) ** 2))
    return (w * np.exp(1j * tilt * p / nx)).astype(dtype)


def add_white_noise(field: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Add circular complex white noise CN(0, sigma^2) (real and imaginary parts
    each N(0, sigma^2/2))."""
    rng = np.random.default_rng(seed)
    s = sigma / math.sqrt(2.0)
    noise = rng.standard_normal(field.shape) * s + 1j * rng.standard_normal(field.shape) * s
    return (field + noise).astype(field.dtype)


def hermite_gaussian_1d(k: int, x: np.ndarray) -> np.ndarray:
    """Normalised 1D Hermite-Gaussian HG_k(x) of Eq. Acc12.

    Evaluated with the three-term recurrence of the normalised Hermite
    functions (psi_0 = pi^-1/4 e^{-x^2/2}, psi_1 = sqrt(2) x psi_0,
    psi_{k+1} = sqrt(2/(k+1)) x psi_k - sqrt(k/(k+1)) psi_{k-1}), which equals
    (2^k k! sqrt(pi))^{-1/2} e^{-x^2/2} H_k(x) without overflowing.
    """
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.zeros_like(x)
    p = math.pi ** -0.25 * np.exp(-0.5 * x * x)
    for n in range(k):
        p_next = math.sqrt(2.0 / (n + 1)) * x * p - math.sqrt(n / (n + 1)) * p_prev
        p_prev, p = p, p_next
    return p


def hg_field(terms, n: int, delta: float) -> np.ndarray:
    """Sampled sum of 2D Hermite-Gaussians HG_{k,l}(x,y) = HG_k(x) HG_l(y)
    (Eq. Acc16) on the centred n x n grid x = m*delta, y = n*delta.

    ``terms`` is a list of (k, l) orders, e.g. [(1, 2), (3, 1)] for g1 of Eq. Acc20.
    """
    x = centered_coords(n) * delta
    out = np.zeros((n, n), dtype=np.complex128)
    for k, l in terms:
        out += np.outer(hermite_gaussian_1d(k, x), hermite_gaussian_1d(l, x))
    return out


def _gyrator(phi: float) -> np.ndarray:
    c, s = math.cos(phi), math.sin(phi)
    sig = np.array([[0.0, 1.0], [1.0, 0.0]])
    eye = np.eye(2)
    return np.block([[c * eye, s * sig], [-s * sig, c * eye]])


def _rotation(phi: float) -> np.ndarray:
    """Rotation of the (x, y) plane by phi: A = D = R(phi), B = C = 0."""
    c, s = math.cos(phi), math.sin(phi)
    r = np.array([[c, -s], [s, c]])
    z = np.zeros((2, 2))
    return np.block([[r, z], [z, r]])


def _sym2(rng, lo, hi) -> np.ndarray:
    a, b, c = rng.uniform(lo, hi, size=3)
    return np.array([[a, b], [b, c]])


def random_symplectic_abcd(seed: int, entry_range=(-0.5, 0.5), min_abs_det_b: float = 0.1,
                           max_tries: int = 1000, middle: str = "rotation_gyrator") -> np.ndarray:
    """Random real 4x4 symplectic ABCD matrix (row-major, Eq. Intro04 layout).

    Built as (I,0;C,I) x middle(phi) x (I,B0;0,I) with C, B0 symmetric, entries
    U(entry_range), phi ~ U(0, pi). The middle factor is, by default, a rotation
    of the (x, y) plane followed by a gyrator, both by phi: a gyrator alone
    gives A = cos(phi) I and a symmetric B, which is the special class of
    Sec. 4.A; the rotation makes A and B general (B non-symmetric), the case
    the CM-CC-CM-CC chain exists for. ``middle`` may also be "gyrator" or
    "rotation". Each factor satisfies Eq. Intro12, hence so does the product.
    Draws are rejected until |det B| >= ``min_abs_det_b`` where B is the
    upper-right block of the product.
    """
    rng = np.random.default_rng(seed)
    eye = np.eye(2)
    zero = np.zeros((2, 2))
    for _ in range(max_tries):
        c = _sym2(rng, *entry_range)
        b0 = _sym2(rng, *entry_range)
        phi = rng.uniform(0, math.pi)
        lower = np.block([[eye, zero], [c, eye]])
        upper = np.block([[eye, b0], [zero, eye]])
        if middle == "gyrator":
            mid = _gyrator(phi)
        elif middle == "rotation":
            mid = _rotation(phi)
        else:
            mid = _rotation(phi) @ _gyrator(phi)
        m = lower @ mid @ upper
        if abs(np.linalg.det(m[:2, 2:])) >= min_abs_det_b:
            return m
    raise RuntimeError("random_symplectic_abcd: no draw met the |det B| bound")
