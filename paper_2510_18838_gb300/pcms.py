"""Thin Python binding of libpcms.so (include/pcms.h): argument marshalling only.

Every call takes CUDA torch tensors, passes their device pointers and the current torch
stream to the C ABI, and raises ``PcmsError`` on a non-OK status. There is no CPU
fallback: if the library has not been built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpcms.so")

OK, INVALID_ARG, UNDERDETERMINED, ILL_CONDITIONED, OUT_OF_MEMORY, TIMEOUT, CUDA_ERR, CAPACITY = range(8)
STATUS_NAMES = ["OK", "INVALID_ARG", "UNDERDETERMINED", "ILL_CONDITIONED", "OUT_OF_MEMORY",
                "TIMEOUT", "CUDA", "CAPACITY"]
FP64, MIXED = 0, 1
WEIGHTS = {"wendland_c2": 0, "gaussian": 1, "c4": 2, "const": 3, "noop": 4, "mq": 5,
           "imq": 6, "tps": 7, "cubic": 8}


class PcmsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{STATUS_NAMES[status] if 0 <= status < 8 else status}] {msg}")
        self.status = status


class MapOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("weight", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("min_neighbors", ctypes.c_int),
                ("domain_known", ctypes.c_int), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("growth", ctypes.c_int)]


class MapInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("basis_degree", ctypes.c_int), ("n_terms", ctypes.c_int),
                ("precision", ctypes.c_int), ("n_src", ctypes.c_int64), ("n_tgt", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("n_underdetermined", ctypes.c_int64),
                ("n_ill_conditioned", ctypes.c_int64), ("max_neighbors", ctypes.c_int64),
                ("max_radius_doublings", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int), ("basis_degree", ctypes.c_int),
                ("radius", ctypes.c_double), ("opts", MapOpts),
                ("src_pts", ctypes.c_void_p), ("n_src", ctypes.c_int64),
                ("tgt_pts", ctypes.c_void_p), ("n_tgt", ctypes.c_int64),
                ("fields", ctypes.c_void_p), ("n_fields", ctypes.c_int),
                ("out", ctypes.c_void_p), ("map_key", ctypes.c_int64), ("reuse_map", ctypes.c_int),
                ("tri", ctypes.c_void_p), ("n_tri", ctypes.c_int64),
                ("elem_ids", ctypes.c_void_p), ("bytes_hint", ctypes.c_int64),
                ("host_io", ctypes.c_int)]


def _host_io(*tensors) -> int:
    """1 if a request's tensors are all host tensors (the server stages them; pin them with
    Tensor.pin_memory() so the copies overlap other requests), 0 if all are CUDA tensors."""
    dev = {t.is_cuda for t in tensors if t is not None}
    if len(dev) != 1:
        raise ValueError("a request's tensors must be all CUDA or all host tensors")
    return 0 if dev.pop() else 1


class RequestResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_end", ctypes.c_double), ("bytes_reserved", ctypes.c_int64),
                ("used_cached_map", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("basis_degree", ctypes.c_int),
                ("radius", ctypes.c_double), ("weight", ctypes.c_int),
                ("src_pts", ctypes.c_void_p), ("n_src", ctypes.c_int64),
                ("tgt_pts", ctypes.c_void_p), ("n_tgt", ctypes.c_int64),
                ("fields", ctypes.c_void_p), ("n_fields", ctypes.c_int),
                ("out", ctypes.c_void_p), ("target_status", ctypes.c_void_p)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("precision", ctypes.c_int),
                ("mode", ctypes.c_int), ("bucket", ctypes.c_int), ("lanes", ctypes.c_int),
                ("cell_div", ctypes.c_double), ("apply_form", ctypes.c_int)]


TUNE_MAP, TUNE_ONESHOT, TUNE_APPLY = 1, 2, 3

BATCH_MAX_POINTS = 131072
BATCH_MAX_ITEMS = 256

REQ_MLS, REQ_MESH = 0, 1

_lib = None

# exported symbol -> (restype, argtypes)
_P, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "pcms_version": (_I, []),
    "pcms_last_error": (ctypes.c_char_p, []),
    "pcms_map_opts_default": (None, [_P]),
    "pcms_create_map": (_I, [_I, _P, _I64, _P, _I64, _I, _D, _P, _P, _P]),
    "pcms_apply_map": (_I, [_P, _P, _I, _P, _P]),
    "pcms_apply_map_noalloc": (_I, [_P, _P, _I, _P, _P]),
    "pcms_apply_map_bf16": (_I, [_P, _P, _I, _P, _P]),
    "pcms_mls_transfer": (_I, [_I, _P, _I64, _P, _I64, _I, _D, _P, _P, _I, _P, _P, _P]),
    "pcms_count_neighbors": (_I, [_I, _P, _I64, _P, _I64, _I, _D, _P, _P, _P, _P, _P]),
    "pcms_mls_transfer_batch": (_I, [_P, _I, _P, _P]),
    "pcms_tune_set": (_I, [_P, _I]),
    "pcms_tune_count": (_I, []),
    "pcms_tune_get": (_I, [_I, _P]),
    "pcms_map_info": (_I, [_P, _P]),
    "pcms_map_export": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "pcms_map_destroy": (None, [_P, _P]),
    "pcms_mesh_create": (_I, [_P, _I64, _P, _I64, _P, _P]),
    "pcms_locate_interp": (_I, [_P, _P, _I64, _P, _P, _P, _P, _P]),
    "pcms_mesh_centroids": (_I, [_P, _P, _P]),
    "pcms_mesh_integrate": (_I, [_P, _P, _P, _P]),
    "pcms_l2_project": (_I, [_P, _P, _P, _P, _D, _I, _P, _P]),
    "pcms_mesh_destroy": (None, [_P, _P]),
    "pcms_server_create": (_I, [_I, _I64, _P]),
    "pcms_server_submit": (_I, [_P, _P, _P]),
    "pcms_server_poll": (_I, [_P, _P, _I, _D, _P]),
    "pcms_server_drain": (_I, [_P, _D]),
    "pcms_server_now": (_D, [_P]),
    "pcms_server_set_batching": (_I, [_P, _I64]),
    "pcms_server_batch_stats": (_I, [_P, _P, _P]),
    "pcms_server_memory": (_I, [_P, _P, _P, _P]),
    "pcms_server_destroy": (None, [_P]),
    "pcms_trace_enable": (_I, [_I]),
    "pcms_trace_count": (_I, []),
    "pcms_trace_get": (_I, [_I, ctypes.c_char_p, _I, _P, _P]),
}


def trace_enable(on: bool = True, count_only: bool = False) -> None:
    """Start (clearing the table) or stop tracing in the library: per-kernel CUDA-event
    timing plus work counts, or with ``count_only`` launch counts alone (no events, no
    extra work, for timed regions)."""
    _check(lib().pcms_trace_enable(0 if not on else (2 if count_only else 1)))


def trace_read() -> dict:
    """{kernel name: (launches, total_ms)} accumulated since the last trace_enable(True)."""
    L = lib()
    out = {}
    for i in range(L.pcms_trace_count()):
        buf = ctypes.create_string_buffer(128)
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(L.pcms_trace_get(i, buf, 128, ctypes.byref(n), ctypes.byref(ms)))
        out[buf.value.decode()] = (int(n.value), float(ms.value))
    return out


def lib():
    """Load libpcms.so (built by ``paper_2510_18838_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpcms.so not built ({LIB_PATH}); run "
                          "`python -m paper_2510_18838_gb300.build` or __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st: int):
    if st != OK:
        msg = lib().pcms_last_error()
        raise PcmsError(st, msg.decode() if msg else "")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


def _req_tensor(t, dtype, shape, name):
    """A serving request's tensor, used in place: the server reads and writes it after
    submit returns, so a copy (to fix its dtype or layout) would not be the caller's."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


GROWTH = {"target": 0, "global": 1}


def make_opts(precision="fp64", weight="wendland_c2", lam=0.0, min_neighbors=0, domain=None,
              growth="target"):
    """pcms_map_opts. growth: "target" (each target doubles its radius) or "global" (one
    shared radius for all targets), used when min_neighbors > 0."""
    o = MapOpts()
    lib().pcms_map_opts_default(ctypes.byref(o))
    o.precision = FP64 if precision == "fp64" else MIXED
    o.weight = WEIGHTS[weight]
    o.lambda_ = float(lam)
    o.min_neighbors = int(min_neighbors)
    o.growth = GROWTH[growth]
    if domain is not None:
        lo, hi = domain
        o.domain_known = 1
        for d in range(len(lo)):
            o.lo[d], o.hi[d] = float(lo[d]), float(hi[d])
    return o


@dataclass
class Map:
    """Cached MLS operator (pcms_create_map). ``apply`` evaluates it on fields."""
    handle: ctypes.c_void_p
    dim: int
    n_src: int
    n_tgt: int
    precision: str
    status_code: int = OK

    @property
    def dtype(self):
        return torch.float64 if self.precision == "fp64" else torch.float32

    def apply(self, fields, out=None, stream=None):
        f = _dev(fields, self.dtype, "fields")
        squeeze = f.dim() == 1
        if squeeze:
            f = f[None]
        nf = f.shape[0]
        if out is None:
            out = torch.empty((nf, self.n_tgt), dtype=self.dtype, device=f.device)
        _check(lib().pcms_apply_map(self.handle, _ptr(f), nf, _ptr(out), _stream(stream)))
        return out[0] if squeeze else out

    def apply_bf16(self, fields, out=None, stream=None):
        """pcms_apply_map_bf16: the apply on the tensor cores (mixed maps, float32 fields)."""
        f = _dev(fields, torch.float32, "fields")
        squeeze = f.dim() == 1
        if squeeze:
            f = f[None]
        nf = f.shape[0]
        if out is None:
            out = torch.empty((nf, self.n_tgt), dtype=torch.float32, device=f.device)
        _check(lib().pcms_apply_map_bf16(self.handle, _ptr(f), nf, _ptr(out), _stream(stream)))
        return out[0] if squeeze else out

    def apply_noalloc(self, fields, out, stream=None):
        """pcms_apply_map_noalloc into a caller tensor (no allocation on any side; usable
        inside CUDA-graph capture). fields [F, n_src] or [n_src], out [F, n_tgt] or [n_tgt],
        both contiguous CUDA tensors of the map's dtype."""
        for t, name in ((fields, "fields"), (out, "out")):
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != self.dtype \
                    or not t.is_contiguous():
                raise TypeError(f"{name} must be a contiguous CUDA {self.dtype} tensor")
        nf = 1 if fields.dim() == 1 else fields.shape[0]
        _check(lib().pcms_apply_map_noalloc(self.handle, _ptr(fields), nf, _ptr(out),
                                            _stream(stream)))
        return out

    def info(self) -> dict:
        i = MapInfo()
        _check(lib().pcms_map_info(self.handle, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in MapInfo._fields_}

    def export(self, stream=None):
        """(offsets int64[nt+1], cols int32[nnz] caller source ids, vals float64[nnz],
        status int8[nt], radius_doublings int32[nt]), rows in caller target order."""
        nnz = self.info()["nnz"]
        dev = torch.device("cuda", torch.cuda.current_device())
        off = torch.empty(self.n_tgt + 1, dtype=torch.int64, device=dev)
        cols = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        vals = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
        st = torch.empty(max(self.n_tgt, 1), dtype=torch.int8, device=dev)
        kx = torch.empty(max(self.n_tgt, 1), dtype=torch.int32, device=dev)
        _check(lib().pcms_map_export(self.handle, _ptr(off), _ptr(cols), _ptr(vals), _ptr(st),
                                     _ptr(kx), _stream(stream)))
        return off, cols[:nnz], vals[:nnz], st[:self.n_tgt], kx[:self.n_tgt]

    def destroy(self, stream=None):
        if self.handle:
            lib().pcms_map_destroy(self.handle, _stream(stream))
            self.handle = None

    def __del__(self):
        try:
            if self.handle and torch.cuda.is_available():
                self.destroy()
        except Exception:
            pass


def create_map(src, tgt, degree, radius, precision="fp64", weight="wendland_c2", lam=0.0,
               min_neighbors=0, domain=None, stream=None, allow_underdetermined=True,
               growth="target") -> Map:
    """pcms_create_map. src/tgt: float64 CUDA tensors [dim, n]."""
    src = _dev(src, torch.float64, "src")
    tgt = _dev(tgt, torch.float64, "tgt")
    dim = src.shape[0]
    o = make_opts(precision, weight, lam, min_neighbors, domain, growth)
    h = ctypes.c_void_p()
    st = lib().pcms_create_map(dim, _ptr(src), src.shape[1], _ptr(tgt), tgt.shape[1], int(degree),
                               float(radius), ctypes.byref(o), _stream(stream), ctypes.byref(h))
    if st != OK and not (st == UNDERDETERMINED and allow_underdetermined and h.value):
        _check(st)
    return Map(h, dim, src.shape[1], tgt.shape[1], precision, st)


def mls_transfer(src, tgt, fields, degree, radius, precision="fp64", weight="wendland_c2",
                 lam=0.0, min_neighbors=0, domain=None, with_status=True, out=None, stream=None,
                 growth="target"):
    """pcms_mls_transfer (one shot, no operator kept). Returns (values [F, nt], status)."""
    src = _dev(src, torch.float64, "src")
    tgt = _dev(tgt, torch.float64, "tgt")
    dt = torch.float64 if precision == "fp64" else torch.float32
    f = _dev(fields, dt, "fields")
    if f.dim() == 1:
        f = f[None]
    nf = f.shape[0]
    nt = tgt.shape[1]
    if out is None:
        out = torch.empty((nf, nt), dtype=dt, device=src.device)
    status = torch.empty(max(nt, 1), dtype=torch.int8, device=src.device) if with_status else None
    o = make_opts(precision, weight, lam, min_neighbors, domain, growth)
    st = lib().pcms_mls_transfer(src.shape[0], _ptr(src), src.shape[1], _ptr(tgt), nt, int(degree),
                                 float(radius), ctypes.byref(o), _ptr(f), nf, _ptr(out),
                                 _ptr(status), _stream(stream))
    if st not in (OK, UNDERDETERMINED):
        _check(st)
    return out, (status[:nt] if status is not None else None)


def tune_set(entries):
    """pcms_tune_set: replace the plan tuning table. entries: dicts with dim, degree,
    precision ("mixed"/"fp64"), mode (TUNE_MAP, TUNE_ONESHOT or TUNE_APPLY), bucket, and
    lanes + cell_div, or apply_form for TUNE_APPLY."""
    arr = (TuneEntry * max(len(entries), 1))()
    for i, e in enumerate(entries):
        x = arr[i]
        x.dim, x.degree = int(e["dim"]), int(e["degree"])
        x.precision = FP64 if e.get("precision", "mixed") == "fp64" else MIXED
        x.mode, x.bucket = int(e["mode"]), int(e["bucket"])
        x.lanes = int(e.get("lanes", 0))
        x.cell_div = float(e.get("cell_div", 0.0))
        x.apply_form = int(e.get("apply_form", 0))
    _check(lib().pcms_tune_set(ctypes.byref(arr), len(entries)))


def tune_get():
    """The plan tuning table as a list of dicts."""
    L = lib()
    out = []
    for i in range(L.pcms_tune_count()):
        x = TuneEntry()
        _check(L.pcms_tune_get(i, ctypes.byref(x)))
        out.append({"dim": x.dim, "degree": x.degree,
                    "precision": "fp64" if x.precision == FP64 else "mixed", "mode": x.mode,
                    "bucket": x.bucket, "lanes": x.lanes, "cell_div": x.cell_div,
                    "apply_form": x.apply_form})
    return out


def mls_transfer_batch(problems, with_status=True, stream=None):
    """pcms_mls_transfer_batch: many small one-shot mixed-precision transfers in one call.
    problems: list of dicts with src [dim, ns] and tgt [dim, nt] (float64, CUDA), fields
    [F, ns] (float32, CUDA), degree, radius and optionally weight. Returns
    (outs, statuses, results): per problem the values [F, nt] and the int8 target statuses
    (or None), and the per-problem pcms_status codes."""
    n = len(problems)
    items = (BatchItem * max(n, 1))()
    keep = []
    outs, stats = [], []
    for i, p in enumerate(problems):
        src = _dev(p["src"], torch.float64, "src")
        tgt = _dev(p["tgt"], torch.float64, "tgt")
        f = _dev(p["fields"], torch.float32, "fields")
        if f.dim() == 1:
            f = f[None]
        nt = tgt.shape[1]
        out = torch.empty((f.shape[0], nt), dtype=torch.float32, device=src.device)
        st = torch.empty(max(nt, 1), dtype=torch.int8, device=src.device) if with_status else None
        it = items[i]
        it.dim, it.basis_degree = src.shape[0], int(p["degree"])
        it.radius = float(p["radius"])
        it.weight = WEIGHTS[p.get("weight", "wendland_c2")]
        it.src_pts, it.n_src = src.data_ptr(), src.shape[1]
        it.tgt_pts, it.n_tgt = tgt.data_ptr(), nt
        it.fields, it.n_fields = f.data_ptr(), f.shape[0]
        it.out = out.data_ptr()
        it.target_status = st.data_ptr() if st is not None else None
        keep += [src, tgt, f]
        outs.append(out)
        stats.append(st[:nt] if st is not None else None)
    res = (ctypes.c_int32 * max(n, 1))()
    _check(lib().pcms_mls_transfer_batch(ctypes.byref(items), n, ctypes.byref(res), _stream(stream)))
    return outs, stats, [int(res[i]) for i in range(n)]


def count_neighbors(src, tgt, radius, degree=1, precision="fp64", weight="wendland_c2",
                    min_neighbors=0, domain=None, with_doublings=False, stream=None,
                    growth="target"):
    """pcms_count_neighbors: per-target neighbour counts (caller order), optionally with the
    radius doublings."""
    src = _dev(src, torch.float64, "src")
    tgt = _dev(tgt, torch.float64, "tgt")
    nt = tgt.shape[1]
    counts = torch.empty(max(nt, 1), dtype=torch.int32, device=src.device)
    kx = torch.empty(max(nt, 1), dtype=torch.int32, device=src.device) if with_doublings else None
    o = make_opts(precision, weight, 0.0, min_neighbors, domain, growth)
    _check(lib().pcms_count_neighbors(src.shape[0], _ptr(src), src.shape[1], _ptr(tgt), nt,
                                      int(degree), float(radius), ctypes.byref(o), _ptr(counts),
                                      _ptr(kx), None, _stream(stream)))
    return (counts[:nt], kx[:nt]) if with_doublings else counts[:nt]


class ProjectionInfo(ctypes.Structure):
    _fields_ = [("intersecting_pairs", ctypes.c_int64), ("iterations", ctypes.c_int),
                ("relative_residual", ctypes.c_double), ("supermesh_area", ctypes.c_double)]


def l2_project(src_mesh, src_field, tgt_mesh, tol=1e-14, max_iter=500, out=None, stream=None):
    """pcms_l2_project: conservative L2 projection of a P1 field (float64 [src vertices])
    onto tgt_mesh's P1 space. Returns (values float64 [tgt vertices], info dict)."""
    f = _dev(src_field, torch.float64, "src_field")
    if out is None:
        out = torch.empty(max(tgt_mesh.n_vertices, 1), dtype=torch.float64, device=f.device)
    info = ProjectionInfo()
    _check(lib().pcms_l2_project(src_mesh.handle, _ptr(f), tgt_mesh.handle, _ptr(out),
                                 float(tol), int(max_iter), ctypes.byref(info), _stream(stream)))
    return out[:tgt_mesh.n_vertices], {k: getattr(info, k) for k, _ in ProjectionInfo._fields_}


class Mesh:
    """Cached triangle mesh + search grid (pcms_mesh_create)."""

    def __init__(self, xy, tri, stream=None):
        xy = _dev(xy, torch.float64, "xy")
        tri = _dev(tri, torch.int32, "tri")
        self.n_vertices = xy.shape[1]
        self.n_tri = tri.shape[1]
        h = ctypes.c_void_p()
        _check(lib().pcms_mesh_create(_ptr(xy), self.n_vertices, _ptr(tri), self.n_tri,
                                      _stream(stream), ctypes.byref(h)))
        self.handle = h

    def locate_interp(self, pts, field=None, with_dim=True, stream=None, elem=None, edim=None,
                      values=None):
        """Returns (elem int32[n], entity_dim int8[n] or None, values float64[n] or None)."""
        pts = _dev(pts, torch.float64, "pts")
        n = pts.shape[1]
        dev = pts.device
        if elem is None:
            elem = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        if with_dim and edim is None:
            edim = torch.empty(max(n, 1), dtype=torch.int8, device=dev)
        if field is not None:
            field = _dev(field, torch.float64, "field")
            if values is None:
                values = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
        _check(lib().pcms_locate_interp(self.handle, _ptr(pts), n, _ptr(field), _ptr(elem),
                                        _ptr(edim) if with_dim else None,
                                        _ptr(values) if field is not None else None,
                                        _stream(stream)))
        return (elem[:n], edim[:n] if with_dim else None,
                values[:n] if field is not None else None)

    def centroids(self, stream=None, out=None):
        """pcms_mesh_centroids: float64 [2, n_tri] triangle centroids."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            out = torch.empty((2, max(self.n_tri, 1)), dtype=torch.float64, device=dev)
        _check(lib().pcms_mesh_centroids(self.handle, _ptr(out), _stream(stream)))
        return out[:, :self.n_tri]

    def integrate(self, field, stream=None) -> float:
        """pcms_mesh_integrate: integral of the piecewise-linear interpolant of a nodal field
        (float64 [n_vertices]) over the mesh; synchronises the stream."""
        f = _dev(field, torch.float64, "field")
        v = ctypes.c_double()
        _check(lib().pcms_mesh_integrate(self.handle, _ptr(f), ctypes.byref(v), _stream(stream)))
        return float(v.value)

    def destroy(self, stream=None):
        if self.handle:
            lib().pcms_mesh_destroy(self.handle, _stream(stream))
            self.handle = None

    def __del__(self):
        try:
            if self.handle and torch.cuda.is_available():
                self.destroy()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (pcms_server_*). Tensors referenced by a submitted
    request are kept alive until the request completes."""

    def __init__(self, n_slots=8, mem_cap_bytes=40 << 30):
        h = ctypes.c_void_p()
        _check(lib().pcms_server_create(int(n_slots), int(mem_cap_bytes), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def now(self) -> float:
        return float(lib().pcms_server_now(self.handle))

    def submit_mls(self, src, tgt, fields, out, degree, radius, precision="mixed",
                   weight="wendland_c2", min_neighbors=0, map_key=-1, reuse=False, bytes_hint=0):
        if src.dim() != 2 or tgt.dim() != 2 or fields.dim() != 2:
            raise ValueError("src, tgt: [dim, n]; fields: [n_fields, n_src]")
        dim, ns, nt, nf = src.shape[0], src.shape[1], tgt.shape[1], fields.shape[0]
        fdt = torch.float32 if precision == "mixed" else torch.float64
        _req_tensor(src, torch.float64, (dim, ns), "src")
        _req_tensor(tgt, torch.float64, (dim, nt), "tgt")
        _req_tensor(fields, fdt, (nf, ns), "fields")
        _req_tensor(out, fdt, (nf, nt), "out")
        r = Request()
        r.kind = REQ_MLS
        r.dim = src.shape[0]
        r.basis_degree = int(degree)
        r.radius = float(radius)
        r.opts = make_opts(precision, weight, 0.0, min_neighbors)
        r.src_pts, r.n_src = src.data_ptr(), src.shape[1]
        r.tgt_pts, r.n_tgt = tgt.data_ptr(), tgt.shape[1]
        r.fields, r.n_fields = fields.data_ptr(), fields.shape[0]
        r.out = out.data_ptr()
        r.map_key = int(map_key)
        r.reuse_map = 1 if reuse else 0
        r.bytes_hint = int(bytes_hint)
        r.host_io = _host_io(src, tgt, fields, out)
        return self._submit(r, (src, tgt, fields, out))

    def submit_mesh(self, xy, tri, pts, field, values, elem, bytes_hint=0):
        if xy.dim() != 2 or tri.dim() != 2 or pts.dim() != 2:
            raise ValueError("xy: [2, n_vertices]; tri: [3, n_triangles]; pts: [2, n]")
        nv, ntri, nt = xy.shape[1], tri.shape[1], pts.shape[1]
        _req_tensor(xy, torch.float64, (2, nv), "xy")
        _req_tensor(tri, torch.int32, (3, ntri), "tri")
        _req_tensor(pts, torch.float64, (2, nt), "pts")
        _req_tensor(elem, torch.int32, (nt,), "elem")
        if (field is None) != (values is None):
            raise ValueError("field and values go together")
        if field is not None:
            _req_tensor(field, torch.float64, (nv,), "field")
            _req_tensor(values, torch.float64, (nt,), "values")
        r = Request()
        r.kind = REQ_MESH
        r.src_pts, r.n_src = xy.data_ptr(), xy.shape[1]
        r.tri, r.n_tri = tri.data_ptr(), tri.shape[1]
        r.tgt_pts, r.n_tgt = pts.data_ptr(), pts.shape[1]
        r.fields = field.data_ptr() if field is not None else None
        r.out = values.data_ptr() if values is not None else None
        r.elem_ids = elem.data_ptr()
        r.bytes_hint = int(bytes_hint)
        r.host_io = _host_io(xy, tri, pts, field, values, elem)
        return self._submit(r, (xy, tri, pts, field, values, elem))

    def _submit(self, r, keep):
        t = ctypes.c_int64()
        _check(lib().pcms_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def poll(self, max_results=256, timeout_s=0.0):
        buf = (RequestResult * max_results)()
        n = ctypes.c_int()
        _check(lib().pcms_server_poll(self.handle, buf, max_results, float(timeout_s),
                                      ctypes.byref(n)))
        out = []
        for i in range(n.value):
            x = buf[i]
            self._keep.pop(x.ticket, None)
            out.append({"ticket": x.ticket, "status": x.status, "t_submit": x.t_submit,
                        "t_start": x.t_start, "t_end": x.t_end, "bytes": x.bytes_reserved,
                        "cached": bool(x.used_cached_map)})
        return out

    def drain(self, timeout_s=600.0):
        _check(lib().pcms_server_drain(self.handle, float(timeout_s)))

    def set_batching(self, max_points: int):
        """Batch one-shot mixed MLS requests of at most max_points points per set (0: off)."""
        _check(lib().pcms_server_set_batching(self.handle, int(max_points)))

    def batch_stats(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pcms_server_batch_stats(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return {"batches": a.value, "batched_requests": b.value}

    def memory(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pcms_server_memory(self.handle, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c)))
        return {"in_use": a.value, "peak": b.value, "cached_maps": c.value}

    def close(self):
        if self.handle:
            lib().pcms_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
