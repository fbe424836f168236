"""The oracle's chain (dense centred DFT sums, Sec. 4.B, Eq. HA28) against the
same chain built from a library FFT (torch.fft on the CPU, in FP64): CC^B as
-(1/(Nx Ny)) IFFT(chi_B FFT(.)) with the chirp over centred bins, CM over
centred samples. The two share no arithmetic but the chirp parameters, so a
wrong sign, index centring or constant in either fails here. The library
chain is the one `bench.py --workload libfft` times for context."""
from __future__ import annotations

import importlib.util
import math
import os

import numpy as np
import pytest

from oracle import nslct_oracle as O
from paper_1707_03688_gb300 import inputs as I

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("nx,ny,seed", [(64, 48, 0), (32, 32, 5), (40, 64, 7), (24, 96, 11)])
def test_oracle_chain_equals_library_fft_chain(nx, ny, seed):
    B = _bench()
    m = I.random_symplectic_abcd(seed)
    params = O.plan(m)
    dx, dy = math.sqrt(2 * math.pi / nx), math.sqrt(2 * math.pi / ny)
    g = I.blob_field(nx, ny, seed=seed)
    ref = O.forward(g, params, dx, dy)
    tabs = B._fft_chain_tables(params, nx, ny, dx, dy, torch.device("cpu"), torch.complex128)
    got = B._fft_chain(torch.from_numpy(g.astype(np.complex128)), tabs).numpy()
    assert O.rel_l2(got, ref) < 1e-12, (nx, ny)


def test_library_fft_chain_catches_a_wrong_chirp_sign():
    """A CM with the opposite sign is far from the oracle's chain."""
    B = _bench()
    nx = ny = 32
    params = O.plan(I.random_symplectic_abcd(5))
    dx = dy = math.sqrt(2 * math.pi / nx)
    g = I.blob_field(nx, ny, seed=5)
    ref = O.forward(g, params, dx, dy)
    chi_h, cm2, chi_b, cm1 = B._fft_chain_tables(params, nx, ny, dx, dy, torch.device("cpu"), torch.complex128)
    got = B._fft_chain(torch.from_numpy(g.astype(np.complex128)), (chi_h, cm2.conj(), chi_b, cm1)).numpy()
    assert O.rel_l2(got, ref) > 1e-2
