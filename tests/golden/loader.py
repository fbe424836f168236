"""Readers for the paper's printed values stored as text fixtures in this folder."""
from __future__ import annotations

import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


def _rows(name):
    with open(os.path.join(_HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            yield [part.strip() for part in line.split("|")]


def paper_matrices():
    """{name: 4x4 ndarray} of the ABCD matrices printed in the paper."""
    out = {}
    for name, _cite, vals in _rows("paper_matrices.txt"):
        out[name] = np.array([float(v) for v in vals.split()]).reshape(4, 4)
    return out


def paper_values():
    """{key: float} of the error figures printed in the paper."""
    return {key: float(val) for key, _cite, val in _rows("paper_values.txt")}
