"""Shared helpers for the parity tests (no method arithmetic here)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcms.h")

# tolerances from the stated accuracy targets: FP64 path 1e-12, mixed path 2e-5,
# measured norm-wise per field (max |gpu - oracle| / max |oracle| over OK targets)
TOL_FP64 = 1e-12
TOL_MIXED = 2e-5


def normwise_err(got, ref, mask=None):
    got = np.atleast_2d(np.asarray(got, dtype=np.float64))
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    assert got.shape == ref.shape, (got.shape, ref.shape)
    if mask is not None:
        got, ref = got[:, mask], ref[:, mask]
    if ref.size == 0:
        return 0.0
    den = np.max(np.abs(ref), axis=1)
    den[den == 0] = 1.0
    return float(np.max(np.max(np.abs(got - ref), axis=1) / den))


def table1_cases():
    """(kind, q, value) rows of tests/golden/table1_weights.txt: the weights of Table 1
    (Sec. 3.2.1) at points where each formula has a closed form, evaluated by hand (the
    derivation is on each row)."""
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "table1_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, q, value = line.split()[:3]
        rows.append((kind, float(q), float(value)))
    return rows


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pcms_[a-z0-9_]+)\s*\(", txt)))


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rows_as_sets(off, cols):
    off = np.asarray(off)
    cols = np.asarray(cols)
    return [np.sort(cols[off[i]:off[i + 1]]) for i in range(len(off) - 1)]
