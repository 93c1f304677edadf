"""FP64 CPU oracle for the PCMS field-transfer hot path (arXiv 2510.18838).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``; the product path never imports it. It shares no
code with the CUDA library. The arithmetic lives in ``pcms_oracle.c`` (plain C, FP64,
compiled with -ffp-contract=off); this module compiles it with gcc on first use and wraps
it with numpy.

Dimensions: MLS in 2 to 5 dimensions (the paper maps fields in up to five, Sec. 1 and
Sec. 5.2's 5D distribution function); the cell-list search (mode="grid") covers 2D and 3D
and falls back to brute force above. Meshes are 2D.

Definitions followed (see the C file for details):
  * radius selection and minimum-count growth -- Sec. 3.2.1, Table 1 (``r > r_c -> 0``);
  * weighted polynomial fit, Tikhonov term, value = c_0 -- Sec. 3.2.1, Eq. 1;
  * RBF weights -- Table 1 (a = 2) plus Wendland C2;
  * point localization with lowest-order classification -- Sec. 3.3;
  * barycentric (parametric) interpolation -- Sec. 3.3.

Parity pins: every function here is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, library routines (numpy lstsq/solve), exact rational arithmetic
(``fractions.Fraction``) and brute force on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcms_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

WEIGHTS = {
    "wendland_c2": 0, "gaussian": 1, "c4": 2, "const": 3, "noop": 4,
    "mq": 5, "imq": 6, "tps": 7, "cubic": 8,
}
STATUS_OK, STATUS_UNDERDETERMINED, STATUS_ILL_CONDITIONED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile pcms_oracle.c into _build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_version.restype = i32
        lib.orc_weight.restype = f64
        lib.orc_weight.argtypes = [i32, f64]
        lib.orc_num_terms.restype = i32
        lib.orc_num_terms.argtypes = [i32, i32]
        lib.orc_set_threads.argtypes = [i32]
        lib.orc_get_threads.restype = i32
        lib.orc_count_neighbors.restype = i64
        lib.orc_count_neighbors.argtypes = [i32, P, i64, P, i64, f64, i32, i32, i32, P, P]
        lib.orc_fill_neighbors.argtypes = [i32, P, i64, P, i64, f64, i32, i32, P, P, P]
        lib.orc_global_doublings.restype = i32
        lib.orc_global_doublings.argtypes = [i32, P, i64, P, i64, f64, i32, i32, i32]
        lib.orc_mls.argtypes = [i32, i32, i32, f64, P, i64, P, i64, P, i32, f64, i32, i32,
                                P, P, P, P, P, P]
        lib.orc_orient2d_sign.restype = i32
        lib.orc_orient2d_sign.argtypes = [f64] * 6
        lib.orc_orient2d_sign_batch.argtypes = [i64, P, P, P, P]
        lib.orc_locate.argtypes = [P, i64, P, i64, P, i64, i32, P, P, P, P]
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def weight(kind: str, q: float) -> float:
    """phi(q), q = r / r_c (Table 1 with a = 2; Wendland C2)."""
    return float(_load().orc_weight(WEIGHTS[kind], float(q)))


def num_terms(dim: int, degree: int) -> int:
    return int(_load().orc_num_terms(dim, degree))


def _need(dim, degree, min_neighbors):
    return max(int(min_neighbors), num_terms(dim, degree)) if min_neighbors > 0 else 0


GROWTH = ("target", "global")


def global_doublings(src, tgt, radius, weight="wendland_c2", min_neighbors=0, degree=1,
                     mode="brute") -> int:
    """Global reading of the Sec. 3.2.1 minimum-count rule: the number of times one radius
    shared by all targets is doubled until every target selects max(min_neighbors, m)
    sources (or all of them). 0 without min_neighbors."""
    lib = _load()
    src, tgt = _f64(src), _f64(tgt)
    dim, ns = src.shape
    need = _need(dim, degree, min_neighbors)
    return int(lib.orc_global_doublings(dim, _p(src), ns, _p(tgt), tgt.shape[1], float(radius),
                                        WEIGHTS[weight], need, 1 if mode == "grid" else 0))


def neighbors(src, tgt, radius, weight="wendland_c2", min_neighbors=0, degree=1,
              mode="brute", growth="target"):
    """Neighbour lists (Sec. 3.2.1 radius selection, ascending source index).
    Returns (offsets int64[nt+1], cols int32[nnz], kexp int32[nt]); kexp[i] is the
    number of radius doublings target i needed (0 without min_neighbors). growth="global"
    uses the single radius radius * 2^K of global_doublings for every target (kexp = K)."""
    if growth not in GROWTH:
        raise ValueError(f"growth must be one of {GROWTH}")
    if growth == "global" and min_neighbors > 0:
        k = global_doublings(src, tgt, radius, weight, min_neighbors, degree, mode)
        off, cols, _ = neighbors(src, tgt, np.ldexp(float(radius), k), weight, 0, degree, mode)
        return off, cols, np.full(np.shape(tgt)[1], k, np.int32)
    lib = _load()
    src, tgt = _f64(src), _f64(tgt)
    dim, ns = src.shape
    nt = tgt.shape[1]
    counts = np.zeros(nt, np.int32)
    kexp = np.zeros(nt, np.int32)
    m = 1 if mode == "grid" else 0
    need = _need(dim, degree, min_neighbors)
    lib.orc_count_neighbors(dim, _p(src), ns, _p(tgt), nt, float(radius), WEIGHTS[weight],
                            need, m, _p(counts), _p(kexp))
    offsets = np.zeros(nt + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    cols = np.zeros(max(int(offsets[-1]), 1), np.int32)
    lib.orc_fill_neighbors(dim, _p(src), ns, _p(tgt), nt, float(radius), WEIGHTS[weight], m,
                           _p(kexp), _p(offsets), _p(cols))
    return offsets, cols[: offsets[-1]], kexp


def mls(src, tgt, fields, degree, radius, weight="wendland_c2", lam=0.0, min_neighbors=0,
        mode="brute", shape=False, growth="target"):
    """MLS transfer by QR (Sec. 3.2.1, Eq. 1). fields: [F, ns] (or [ns]).
    Returns dict(values float64[F, nt], status int8[nt], kexp int32[nt]) and, with
    shape=True, also offsets, cols (ascending) and shape float64[nnz]. growth="global":
    every target is fitted at the shared radius radius * 2^K of global_doublings."""
    if growth not in GROWTH:
        raise ValueError(f"growth must be one of {GROWTH}")
    if growth == "global" and min_neighbors > 0:
        k = global_doublings(src, tgt, radius, weight, min_neighbors, degree, mode)
        out = mls(src, tgt, fields, degree, np.ldexp(float(radius), k), weight, lam, 0, mode,
                  shape)
        out["kexp"][:] = k
        return out
    lib = _load()
    src, tgt = _f64(src), _f64(tgt)
    fields = _f64(fields)
    if fields.ndim == 1:
        fields = fields[None, :]
    fields = np.ascontiguousarray(fields)
    dim, ns = src.shape
    nt = tgt.shape[1]
    nf = fields.shape[0]
    values = np.empty((nf, nt), np.float64)
    status = np.zeros(nt, np.int8)
    kexp = np.zeros(nt, np.int32)
    m = 1 if mode == "grid" else 0
    need = _need(dim, degree, min_neighbors)
    offsets = cols = shp = None
    if shape:
        offsets, _, _ = neighbors(src, tgt, radius, weight, min_neighbors, degree, mode)
        cols = np.zeros(max(int(offsets[-1]), 1), np.int32)
        shp = np.zeros(max(int(offsets[-1]), 1), np.float64)
    lib.orc_mls(dim, degree, WEIGHTS[weight], float(lam), _p(src), ns, _p(tgt), nt,
                _p(fields), nf, float(radius), need, m, _p(values), _p(status), _p(kexp),
                _p(offsets), _p(cols), _p(shp))
    out = dict(values=values, status=status, kexp=kexp)
    if shape:
        nnz = int(offsets[-1])
        out.update(offsets=offsets, cols=cols[:nnz], shape=shp[:nnz])
    return out


def orient2d_sign(a, b, c):
    """Exact sign of (ax-cx)(by-cy) - (ay-cy)(bx-cx). Scalars (tuples) or [2, n] arrays."""
    lib = _load()
    a_arr = np.asarray(a, dtype=np.float64)
    if a_arr.ndim == 1 and a_arr.shape[0] == 2:
        return int(lib.orc_orient2d_sign(*[float(v) for v in (*a, *b, *c)]))
    a_arr, b_arr, c_arr = _f64(a), _f64(b), _f64(c)
    n = a_arr.shape[1]
    out = np.zeros(n, np.int8)
    lib.orc_orient2d_sign_batch(n, _p(a_arr), _p(b_arr), _p(c_arr), _p(out))
    return out


def locate(xy, tri, pts, field=None, mode="exhaustive"):
    """Point localization + barycentric interpolation (Sec. 3.3).
    Returns (elem int32[q], dim int8[q], values float64[q] or None)."""
    lib = _load()
    xy = _f64(xy)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    pts = _f64(pts)
    nv = xy.shape[1]
    ntri = tri.shape[1]
    q = pts.shape[1]
    elem = np.empty(q, np.int32)
    dimc = np.empty(q, np.int8)
    vals = None
    fld = None
    if field is not None:
        fld = _f64(field)
        vals = np.empty(q, np.float64)
    lib.orc_locate(_p(xy), nv, _p(tri), ntri, _p(pts), q, 1 if mode == "grid" else 0,
                   _p(fld), _p(elem), _p(dimc), _p(vals))
    return elem, dimc, vals


from oracle.roundtrip import centroids, p1_integral, round_trip  # noqa: E402,F401
from oracle.projection import l2_projection  # noqa: E402,F401
