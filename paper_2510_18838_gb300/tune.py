"""Plan autotuner for the MLS transfer: measures launch-plan candidates on seeded synthetic
problems on the current GPU and loads the fastest into the library's tuning table
(pcms_tune_set), keyed as the library looks plans up: (dimension, basis degree, precision,
mode, bucket = floor(log2 of the expected neighbour count)).

Candidates per key: lanes per target (8 or 32) x the grid's cell divisor (cell edge =
radius / d; d in 2, 3, 4, 6 in 2D and 1.5, 2, 3 in 3D). Each candidate is timed with CUDA
events (best of `reps`, after one untimed run) on the whole call it affects: a one-shot
transfer (one field) for PCMS_TUNE_ONESHOT keys, operator creation plus a multi-field apply
for PCMS_TUNE_MAP keys. A key gets an entry only where the best candidate beats the plan
rules' own choice by more than `margin`, so the table never replaces a rule with a slower
plan as measured. For the apply, the CUDA-core and the tensor-core forms are timed per field
count on one 3D operator. The table can be saved to and loaded from JSON.
"""
from __future__ import annotations

import json
import math
import time
from dataclasses import asdict, dataclass

import numpy as np
import torch

from . import pcms

DIVS = {2: (2.0, 3.0, 4.0, 6.0), 3: (1.5, 2.0, 3.0)}
LANES = (8, 32)


@dataclass(frozen=True)
class Shape:
    dim: int
    degree: int
    mode: str        # "oneshot" or "map"
    k: float         # expected neighbours per target
    n: int           # sources = targets
    nf: int = 1      # fields (map mode)
    seed: int = 0


def default_shapes(n: int = 400_000) -> list[Shape]:
    """The serving stream's range: 2D and 3D, linear and quadratic, one-shot and operator
    requests, expected neighbour counts 12 to 300 (buckets 3 to 8)."""
    out = []
    for dim in (2, 3):
        for degree in (1, 2):
            for mode in ("oneshot", "map"):
                for k in (12.0, 24.0, 48.0, 96.0, 192.0, 300.0):
                    out.append(Shape(dim, degree, mode, k, n, nf=1 if mode == "oneshot" else 8,
                                     seed=1000 * dim + 100 * degree + int(k)))
    return out


def expected_count(src: np.ndarray, radius: float) -> float:
    """The library's expected neighbour count: sources per box volume times the ball."""
    dim = src.shape[0]
    vol = 1.0
    for d in range(dim):
        vol *= max(float(src[d].max() - src[d].min()), radius)
    ball = math.pi * radius ** 2 if dim == 2 else 4.0 / 3.0 * math.pi * radius ** 3
    return src.shape[1] * ball / vol


def bucket(mean: float) -> int:
    return 0 if mean < 1.0 else min(30, int(math.floor(math.log2(mean))))


def _problem(sh: Shape, device):
    rng = np.random.default_rng(sh.seed)
    src = rng.uniform(0.0, 1.0, (sh.dim, sh.n))
    tgt = rng.uniform(0.0, 1.0, (sh.dim, sh.n))
    ball = math.pi if sh.dim == 2 else 4.0 / 3.0 * math.pi
    radius = (sh.k / (ball * sh.n)) ** (1.0 / sh.dim)
    f = rng.standard_normal((sh.nf, sh.n)).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return t(src), t(tgt), t(f), radius, bucket(expected_count(src, radius))


def _call(sh: Shape, prob):
    src, tgt, f, radius, _ = prob
    if sh.mode == "oneshot":
        out, _ = pcms.mls_transfer(src, tgt, f, sh.degree, radius, precision="mixed",
                                   with_status=False)
        return out
    m = pcms.create_map(src, tgt, sh.degree, radius, precision="mixed")
    out = m.apply(f)
    m.destroy()
    return out


def time_call(fn, reps: int) -> float:
    """best of reps, in ms, CUDA events on the current stream (one untimed run first)"""
    fn()
    torch.cuda.synchronize()
    best = math.inf
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def key_of(sh: Shape, b: int) -> dict:
    return {"dim": sh.dim, "degree": sh.degree, "precision": "mixed",
            "mode": pcms.TUNE_ONESHOT if sh.mode == "oneshot" else pcms.TUNE_MAP, "bucket": b}


def tune(shapes: list[Shape] | None = None, reps: int = 3, margin: float = 0.05,
         apply_fields=(2, 4, 8, 16), apply_n: int = 200_000, device=None) -> dict:
    """Measure and load the tuning table; returns {"entries": [...], "measurements": [...],
    "seconds": ...}. Keys shared by several shapes keep the first shape's result."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    shapes = default_shapes() if shapes is None else shapes
    t_start = time.perf_counter()
    entries: list[dict] = []
    done = set()
    meas = []
    for sh in shapes:
        prob = _problem(sh, device)
        key = key_of(sh, prob[4])
        kt = tuple(sorted(key.items()))
        if kt in done:
            continue
        done.add(kt)
        pcms.tune_set(entries)
        rule = time_call(lambda: _call(sh, prob), reps)
        cands = {}
        for lanes in LANES:
            for div in DIVS[sh.dim]:
                pcms.tune_set(entries + [dict(key, lanes=lanes, cell_div=div)])
                cands[(lanes, div)] = time_call(lambda: _call(sh, prob), reps)
        best = min(cands, key=cands.get)
        meas.append({"shape": asdict(sh), "key": key, "rule_ms": rule,
                     "best": {"lanes": best[0], "cell_div": best[1], "ms": cands[best]},
                     "candidates_ms": {f"{l}x{d}": v for (l, d), v in cands.items()}})
        if cands[best] < (1.0 - margin) * rule:
            entries.append(dict(key, lanes=best[0], cell_div=best[1]))
        del prob
    # the apply form per field count, on one 3D quadratic operator (57 neighbours)
    rng = np.random.default_rng(77)
    src = torch.from_numpy(rng.uniform(0, 1, (3, apply_n))).to(device)
    tgt = torch.from_numpy(rng.uniform(0, 1, (3, apply_n))).to(device)
    radius = (57.0 / (4.0 / 3.0 * math.pi * apply_n)) ** (1.0 / 3.0)
    pcms.tune_set(entries)
    m = pcms.create_map(src, tgt, 2, radius, precision="mixed")
    for nf in apply_fields:
        f = torch.from_numpy(rng.standard_normal((nf, apply_n)).astype(np.float32)).to(device)
        t_cc = time_call(lambda: m.apply(f), reps)
        t_tc = time_call(lambda: m.apply_bf16(f), reps)
        meas.append({"apply_fields": nf, "cuda_core_ms": t_cc, "tensor_core_ms": t_tc})
        if t_tc < (1.0 - margin) * t_cc:
            for deg in (1, 2):
                for dim in (2, 3):
                    entries.append({"dim": dim, "degree": deg, "precision": "mixed",
                                    "mode": pcms.TUNE_APPLY, "bucket": nf, "apply_form": 1})
    m.destroy()
    pcms.tune_set(entries)
    return {"entries": entries, "measurements": meas, "seconds": time.perf_counter() - t_start,
            "device": torch.cuda.get_device_name(device)}


def save(table: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1)


def load(path: str) -> dict:
    """Load a saved table into the library (it was measured on some GPU; re-tune on another)."""
    with open(path) as f:
        table = json.load(f)
    pcms.tune_set(table["entries"])
    return table
