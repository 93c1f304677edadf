"""Serving driver: replays a stream of transfer requests through the library's native
continuous-batching server (pcms_server_*) and reports throughput and latency.

Requests come from ``workloads.request_stream`` (Poisson arrivals; point counts log-uniform
in 1k..2M; 2D/3D MLS with linear or quadratic basis and 1..16 fields, 30% of MLS requests
reusing an earlier request's operator; 2D mesh transfers on jittered grids). Their inputs are
synthesised on the device with seeded generators before any timing starts, so every input
is resident in HBM.

Two forms are measured on the same requests:
  served  -- mixed precision, continuous batching: n_slots concurrent requests on their own
             streams, admission under a device-memory cap, cached operators for reuse;
  plain   -- FP64, one request at a time, no caching (each request builds its own operator).
"""
from __future__ import annotations

import math
import statistics
import time
from dataclasses import dataclass, field

import torch

from . import pcms
from . import workloads as W


@dataclass
class DeviceRequest:
    req: W.Request
    tensors: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return self.req.n_tgt


def _rand(gen, shape, device):
    return torch.rand(shape, generator=gen, device=device, dtype=torch.float64)


def _trig_fields_dev(pts, n_fields, seed, max_deg=2):
    """Random trigonometric fields of degree <= max_deg (float32 [F, n]) on the device."""
    dim = pts.shape[0]
    terms = [t for t in __import__("itertools").product(range(max_deg + 1), repeat=dim)
             if sum(t) <= max_deg]
    g = torch.Generator(device="cpu").manual_seed(seed)
    coef = torch.randn((n_fields, 2 * len(terms)), generator=g, dtype=torch.float64)
    coef = (coef / math.sqrt(len(terms))).to(pts.device)
    out = torch.zeros((n_fields, pts.shape[1]), dtype=torch.float64, device=pts.device)
    for i, t in enumerate(terms):
        ph = 2 * math.pi * sum(t[d] * pts[d] for d in range(dim))
        out += coef[:, 2 * i:2 * i + 1] * torch.cos(ph)[None] + coef[:, 2 * i + 1:2 * i + 2] * torch.sin(ph)[None]
    return out.to(torch.float32).contiguous()


def _mesh_dev(n, seed, device):
    """Jittered n x n grid mesh (same construction as workloads.jittered_grid_mesh)."""
    h = 1.0 / n
    g = torch.Generator(device=device).manual_seed(seed)
    idx = torch.arange(n + 1, device=device, dtype=torch.float64)
    y, x = torch.meshgrid(idx * h, idx * h, indexing="ij")
    x, y = x.reshape(-1).clone(), y.reshape(-1).clone()
    nv = (n + 1) * (n + 1)
    rad = 0.3 * h * torch.sqrt(torch.rand(nv, generator=g, device=device, dtype=torch.float64))
    ang = 2 * math.pi * torch.rand(nv, generator=g, device=device, dtype=torch.float64)
    ii = torch.arange(nv, device=device) % (n + 1)
    jj = torch.arange(nv, device=device) // (n + 1)
    inner = (ii > 0) & (ii < n) & (jj > 0) & (jj < n)
    x = torch.where(inner, x + rad * torch.cos(ang), x)
    y = torch.where(inner, y + rad * torch.sin(ang), y)
    xy = torch.stack([x, y]).contiguous()
    ci = torch.arange(n * n, device=device, dtype=torch.int64)
    i, j = ci % n, ci // n
    v00 = j * (n + 1) + i
    tri = torch.empty((3, 2 * n * n), dtype=torch.int32, device=device)
    tri[0, 0::2], tri[1, 0::2], tri[2, 0::2] = v00, v00 + 1, v00 + n + 2
    tri[0, 1::2], tri[1, 1::2], tri[2, 1::2] = v00, v00 + n + 2, v00 + n + 1
    return xy, tri


OUTPUT_KEYS = ("out", "values", "elem")


def to_host(dreqs, pin: bool = False) -> list[DeviceRequest]:
    """The same requests with host copies of their inputs and host output buffers:
    submitted as they are, the server stages every copy on the request's slot stream (host
    I/O requests). Ordinary (pageable) memory by default, as a caller's arrays usually are;
    pin=True page-locks them. Requests sharing a geometry share its host copy."""
    copies = {}
    out = []
    for d in dreqs:
        h = {}
        for k, v in d.tensors.items():
            if k in OUTPUT_KEYS:
                h[k] = torch.empty(v.shape, dtype=v.dtype, pin_memory=pin)
            else:
                key = (v.data_ptr(), v.numel(), v.dtype)
                if key not in copies:
                    c = v.to("cpu")
                    copies[key] = c.pin_memory() if pin else c
                h[k] = copies[key]
        out.append(DeviceRequest(d.req, h))
    return out


def materialize(reqs, device) -> list[DeviceRequest]:
    """Synthesise every request's inputs and outputs on the device (seeded)."""
    out: list[DeviceRequest] = []
    by_id = {}
    for r in reqs:
        d = DeviceRequest(r)
        g = torch.Generator(device=device).manual_seed(r.seed)
        if r.kind == "mesh":
            xy, tri = _mesh_dev(r.mesh_n, r.seed, device)
            d.tensors = dict(xy=xy, tri=tri, field=(xy[0] ** 2 + 3 * xy[0] * xy[1]).contiguous(),
                             pts=_rand(g, (2, r.n_tgt), device),
                             values=torch.empty(r.n_tgt, dtype=torch.float64, device=device),
                             elem=torch.empty(r.n_tgt, dtype=torch.int32, device=device))
        else:
            if r.reuse_of >= 0:
                base = by_id[r.reuse_of].tensors
                src, tgt = base["src"], base["tgt"]
            else:
                src = _rand(g, (r.dim, r.n_src), device)
                tgt = _rand(g, (r.dim, r.n_tgt), device)
            d.tensors = dict(src=src, tgt=tgt,
                             fields=_trig_fields_dev(src, r.n_fields, 1000 + 37 * r.rid),
                             out=torch.empty((r.n_fields, r.n_tgt), dtype=torch.float32,
                                             device=device))
        by_id[r.rid] = d
        out.append(d)
    if torch.device(device).type == "cuda":
        torch.cuda.synchronize()
    return out


def map_key(r: W.Request) -> int:
    """operator cache key: the request that first built the geometry"""
    return r.reuse_of if r.reuse_of >= 0 else r.rid


def submit(server: pcms.Server, d: DeviceRequest, reused_keys: set):
    r, t = d.req, d.tensors
    if r.kind == "mesh":
        return server.submit_mesh(t["xy"], t["tri"], t["pts"], t["field"], t["values"], t["elem"])
    key = map_key(r)
    keep = key in reused_keys
    return server.submit_mls(t["src"], t["tgt"], t["fields"], t["out"], r.degree, r.radius,
                             precision="mixed", map_key=key if keep else -1,
                             reuse=r.reuse_of >= 0)


def run_served(dreqs, n_slots=8, mem_cap=40 << 30, arrivals=None, timeout_s=900.0,
               batch_max=None):
    """Replay through a fresh server. arrivals=None: every request is submitted at once
    (closed loop); else arrival offsets in seconds (open loop). batch_max: the server's
    batching bound in points (None: the library default, 0: no batching). Returns a stats
    dict."""
    reused = {r.req.reuse_of for r in dreqs if r.req.kind == "mls" and r.req.reuse_of >= 0}
    server = pcms.Server(n_slots=n_slots, mem_cap_bytes=mem_cap)
    if batch_max is not None:
        server.set_batching(batch_max)
    torch.cuda.synchronize()
    t_begin = server.now()
    results = {}
    ticket_of = {}
    i = 0
    n = len(dreqs)
    while i < n or len(results) < n:
        now = server.now() - t_begin
        while i < n and (arrivals is None or arrivals[i] <= now):
            tk = submit(server, dreqs[i], reused)
            ticket_of[tk] = i
            i += 1
        wait = 0.0005 if i < n else 0.05
        for res in server.poll(512, timeout_s=wait):
            results[ticket_of[res["ticket"]]] = res
        if server.now() - t_begin > timeout_s:
            raise TimeoutError("serving stream did not finish")
    t_end = max(r["t_end"] for r in results.values())
    mem = server.memory()
    bst = server.batch_stats()
    server.close()
    lat = []
    bad = 0
    for k, res in results.items():
        if res["status"] != pcms.OK:
            bad += 1
        arr = t_begin + (arrivals[k] if arrivals is not None else 0.0)
        lat.append(res["t_end"] - max(arr, res["t_submit"]) if arrivals is not None
                   else res["t_end"] - res["t_submit"])
    pts = sum(d.points for d in dreqs)
    wall = t_end - t_begin
    return dict(points=pts, seconds=wall, points_per_s=pts / wall,
                p50_ms=1e3 * statistics.median(lat), p99_ms=1e3 * _pct(lat, 99),
                failed=bad, cached_hits=sum(1 for r in results.values() if r["cached"]),
                peak_bytes=mem["peak"], batches=bst["batches"],
                batched_requests=bst["batched_requests"], results=[results[i] for i in range(n)])


def run_plain_fp64(dreqs, arrivals=None):
    """FP64, one request at a time, no cache: per-request time and, with arrivals, the
    latency a single-queue server of this form would give."""
    stream = torch.cuda.current_stream()
    durs = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d in dreqs:
        r, t = d.req, d.tensors
        a = time.perf_counter()
        if r.kind == "mesh":
            mesh = pcms.Mesh(t["xy"], t["tri"])
            mesh.locate_interp(t["pts"], t["field"], with_dim=False, elem=t["elem"],
                               values=t["values"])
            mesh.destroy()
        else:
            f64 = t["fields"].to(torch.float64)
            m = pcms.create_map(t["src"], t["tgt"], r.degree, r.radius, precision="fp64")
            m.apply(f64)
            m.destroy()
        stream.synchronize()
        durs.append(time.perf_counter() - a)
    wall = time.perf_counter() - t0
    pts = sum(d.points for d in dreqs)
    out = dict(points=pts, seconds=wall, points_per_s=pts / wall,
               p50_ms=1e3 * statistics.median(durs), p99_ms=1e3 * _pct(durs, 99))
    if arrivals is not None:
        clock, lat = 0.0, []
        for a, s in zip(arrivals, durs):
            clock = max(clock, a) + s
            lat.append(clock - a)
        out.update(queued_p50_ms=1e3 * statistics.median(lat), queued_p99_ms=1e3 * _pct(lat, 99))
    return out


def _pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = (len(xs) - 1) * p / 100.0
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)
