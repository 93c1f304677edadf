"""Benchmark of the GB300 field-transfer hot path (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload serve|transfer]

Workloads (synthetic, seeded; shaped like the paper's field-transfer workloads):
  transfer -- one step = the whole hot path over one batch:
              (a) 2D mesh transfer: 512x512 jittered grid (524,288 triangles), search-grid
                  build + localisation + barycentric interpolation of 1,000,000 points;
              (b) 2D MLS, mixed precision, one-shot: 4M Gaussian-mixture sources -> 4M
                  uniform targets, quadratic basis, Wendland C2, r = 0.01, min 10
                  neighbours (radius doubling);
              (c) 3D MLS, mixed precision: 8M sources (uniform + dense slab) -> 8M targets,
                  quadratic basis, r = 0.012: operator build + apply of 16 fields.
              value = target points mapped per second (1M + 4M + 8M per step).
  serve    -- see paper_2510_18838_gb300/serve.py (continuous-batching request loop).

Timing: W untimed warm-up steps; K timed steps, each bracketed by CUDA events on the
stream the library launches on, with a 256 MiB L2-flushing write between steps (outside
the events); barrier + synchronize on both sides; max over ranks. SM clocks and throttle
reasons are sampled with nvidia-smi during the timed steps. Per-kernel times come from
the library's own CUDA-event tracing on its launching stream.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("target points mapped/sec (MLS + mesh interp) at ≤2e-5 rel err; "
          "p50/p99 request latency")

# ------------------------------------------------------------------------------------
# algorithmic work models (per selected pair / per point); see the design doc
# ------------------------------------------------------------------------------------


def mono_count(dim, deg):
    return math.comb(dim + deg, deg)


def mls_pair_flops(dim, deg, fused_fields):
    """FP32 flops the weighted-moment formulation needs per selected pair: squared
    distance, q, Wendland C2, scaled offsets, moments of degree <= 2k, and (one-shot mode)
    the right-hand side for each field."""
    nm = mono_count(dim, 2 * deg)
    m = mono_count(dim, deg)
    f = (2 * dim - 1) + 2 + 6 + dim + (2 * nm - 1)
    f += fused_fields * (2 * m + 1)
    return f


def spmm_bytes(nnz, ns, nt, nf, elem=4):
    """HBM bytes one apply launch must move at least: column index + value per nonzero,
    every source field row once, every target output row once."""
    return nnz * (4 + elem) + ns * nf * elem + nt * nf * elem


# ------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[3], p[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for n, v in zip(names, r[3]):
                if v.lower() == "active":
                    seen.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "samples": len(rows),
                "reasons": sorted(seen)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------------------------
# transfer workload
# ------------------------------------------------------------------------------------
class TransferWorkload:
    name = ("transfer_mix: mesh 512x512 jittered (524,288 tri) 1M pts + MLS2D mixed 4M->4M "
            "gauss8 quadratic r=0.01 minnb=10 + MLS3D mixed 8M->8M slab quadratic r=0.012 16 fields")

    def __init__(self, torch, pcms, W, device):
        self.torch, self.P, self.W = torch, pcms, W
        self.dev = device
        np = __import__("numpy")
        self.np = np
        c2 = W.mesh_2d()
        c3 = W.mls_2d_gaussian()
        c4 = W.mls_3d_slab()
        self.host = {
            "xy": c2.xy, "tri": c2.tri, "mfield": c2.field, "mpts": c2.pts,
            "s3": c3.src, "t3": c3.tgt, "f3": c3.fields.astype(np.float32),
            "s4": c4.src, "t4": c4.tgt, "f4": c4.fields,
        }
        self.cfg = {"c2": c2, "c3": c3, "c4": c4}
        self.d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in self.host.items()}
        self.points_per_step = c2.pts.shape[1] + c3.tgt.shape[1] + c4.tgt.shape[1]
        self.parts = {}
        self.out = {}
        # work counts for the roofline models
        m4 = pcms.create_map(self.d["s4"], self.d["t4"], 2, c4.radius, precision="mixed")
        self.nnz4 = m4.info()["nnz"]
        m4.destroy()
        cnt = pcms.count_neighbors(self.d["s3"], self.d["t3"], c3.radius, degree=2,
                                   min_neighbors=c3.min_neighbors, precision="mixed")
        self.pairs3 = int(cnt.sum().item())
        torch.cuda.synchronize()

    def step(self, d=None, timed_parts=False):
        P, torch = self.P, self.torch
        d = d or self.d
        c3, c4 = self.cfg["c3"], self.cfg["c4"]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if timed_parts else None
        if ev: ev[0].record()
        mesh = P.Mesh(d["xy"], d["tri"])
        elem, _, vals = mesh.locate_interp(d["mpts"], d["mfield"], with_dim=False)
        if ev: ev[1].record()
        out3, _ = P.mls_transfer(d["s3"], d["t3"], d["f3"], 2, c3.radius, precision="mixed",
                                 min_neighbors=c3.min_neighbors, with_status=False)
        if ev: ev[2].record()
        m4 = P.create_map(d["s4"], d["t4"], 2, c4.radius, precision="mixed")
        out4 = m4.apply(d["f4"])
        m4.destroy()
        mesh.destroy()
        if ev:
            ev[3].record()
            torch.cuda.synchronize()
            self.parts = {"mesh_1M_ms": ev[0].elapsed_time(ev[1]),
                          "mls2d_4M_ms": ev[1].elapsed_time(ev[2]),
                          "mls3d_8M_16f_ms": ev[2].elapsed_time(ev[3])}
        self.out = {"elem": elem, "vals": vals, "out3": out3, "out4": out4}
        return self.points_per_step

    def e2e_step(self, pinned):
        """inputs copied from pinned host buffers, outputs read back, inside the region"""
        torch = self.torch
        d = {k: v.to(self.dev, non_blocking=True) for k, v in pinned.items()}
        self.step(d)
        outs = [self.out["elem"], self.out["vals"], self.out["out3"], self.out["out4"]]
        host = [o.to("cpu") for o in outs]
        torch.cuda.synchronize()
        return sum(o.numel() * o.element_size() for o in host)

    def pinned_inputs(self):
        return {k: v.cpu().pin_memory() for k, v in self.d.items()}

    def input_bytes(self):
        return sum(v.numel() * v.element_size() for v in self.d.values())

    def roofline(self, trace, peaks, kind):
        """dominant kernel of the step and its roofline entry"""
        if not trace:
            return None, None
        name = max(trace, key=lambda k: trace[k][1])
        launches, ms = trace[name]
        avg_s = ms / launches / 1e3
        c3, c4 = self.cfg["c3"], self.cfg["c4"]
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        r = None
        if name == "mls_assemble_fused_mixed":
            fl = self.pairs3 * mls_pair_flops(2, 2, 1)
            r = {"bound": "alu", "achieved": fl / avg_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s"}
        elif name == "mls_assemble_map_mixed":
            fl = self.nnz4 * mls_pair_flops(3, 2, 0)
            r = {"bound": "alu", "achieved": fl / avg_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s"}
        elif name == "apply_spmm":
            by = spmm_bytes(self.nnz4, c4.src.shape[1], c4.tgt.shape[1], 16)
            r = {"bound": "hbm", "achieved": by / avg_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
        if r is not None:
            r["frac"] = r["achieved"] / r["peak"]
            r["traffic"] = None
            r["kernel"] = name
            r["peak_source"] = kind if r["unit"] == "GB/s" else f"{kind} max SM clock x 152 SM x 128 FP32 lanes x 2"
            r["avg_launch_ms"] = ms / launches
        return name, r

    def cpu_sample(self, orc, budget_s=15.0):
        """the oracle as it stands on a bounded, seeded sample of the same workload"""
        np = self.np
        rng = np.random.default_rng(7)
        c2, c3, c4 = self.cfg["c2"], self.cfg["c3"], self.cfg["c4"]
        n2, n3, n4 = 100_000, 1_000, 10_000
        i2 = rng.choice(c2.pts.shape[1], n2, replace=False)
        i3 = rng.choice(c3.tgt.shape[1], n3, replace=False)
        i4 = rng.choice(c4.tgt.shape[1], n4, replace=False)
        t = time.perf_counter()
        orc.locate(c2.xy, c2.tri, c2.pts[:, i2], field=c2.field, mode="grid")
        orc.mls(c3.src, c3.tgt[:, i3], c3.fields, 2, c3.radius, min_neighbors=c3.min_neighbors,
                mode="grid")
        orc.mls(c4.src, c4.tgt[:, i4], c4.fields.astype(np.float64), 2, c4.radius, mode="grid")
        dt = time.perf_counter() - t
        n = n2 + n3 + n4
        return n / dt, n, dt, (f"{n2} mesh points + {n3} MLS2D targets + {n4} MLS3D targets "
                               f"(16 fields), uniform sample, oracle grid mode")


# ------------------------------------------------------------------------------------
def flush_l2(torch, buf):
    buf.add_(1.0)


def run_reference(args, rank, world):
    """The CPU oracle as it stands, on the host cores, on bounded samples (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2510_18838_gb300 import workloads as W
    oracle.build()
    cores = oracle.get_threads()

    class _Stub:
        pass
    wl = TransferWorkload.__new__(TransferWorkload)
    wl.np = np
    wl.cfg = {"c2": W.mesh_2d(), "c3": W.mls_2d_gaussian(), "c4": W.mls_3d_slab()}
    vals = []
    for i in range(args.warmup + args.steps):
        v, n, dt, sample = wl.cpu_sample(oracle)
        if i >= args.warmup:
            vals.append((v, n, dt))
    v = statistics.median(x[0] for x in vals)
    ms = statistics.median(x[2] for x in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": TransferWorkload.name, "sample": sample},
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": "points/s", "cores": cores,
                             "sample": sample},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="transfer", choices=["transfer", "serve"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2510_18838_gb300 import build as B
    B.build()
    from paper_2510_18838_gb300 import pcms
    from paper_2510_18838_gb300 import workloads as W
    dev = torch.device("cuda", local)

    wl = TransferWorkload(torch, pcms, W, dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    pcms.trace_enable(True)
    step_ms = []
    points = 0
    stream = torch.cuda.current_stream()
    for _ in range(args.steps):
        flush_l2(torch, flush)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        points += wl.step()
        b.record(stream)
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
    pcms.trace_enable(False)
    trace = pcms.trace_read()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    torch.cuda.synchronize()
    value = points * world / (total_ms / 1e3)
    wl.step(timed_parts=True)
    parts = dict(wl.parts)

    # end to end: pinned host inputs -> device, the same C-ABI calls, results -> host
    pinned = wl.pinned_inputs()
    e2e_ms = []
    bo = 0
    for i in range(max(2, args.steps)):
        flush_l2(torch, flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bo = wl.e2e_step(pinned)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_med = statistics.median(e2e_ms[1:] if len(e2e_ms) > 2 else e2e_ms)
    bi = wl.input_bytes()

    peaks, kind = measured_peaks()
    kname, roof = wl.roofline(trace, peaks, kind)
    launches = sum(v[0] for v in trace.values())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        v, n, dt, sample = wl.cpu_sample(oracle)
        cpu = {"value": v, "unit": "points/s", "cores": oracle.get_threads(), "kind": "oracle",
               "sample": sample, "seconds": dt}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": wl.name, "points_per_step": wl.points_per_step,
                       "l2": "256 MiB write between timed steps; inputs > L2",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk,
            "e2e": {"value": wl.points_per_step / (e2e_med / 1e3), "unit": "points/s",
                    "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                    "ms_per_step": e2e_med},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "parts_ms": parts,
            "kernels_ms": {k: round(v[1] / args.steps, 4) for k, v in
                           sorted(trace.items(), key=lambda kv: -kv[1][1])},
            "work": {"mls2d_pairs": wl.pairs3, "mls3d_nnz": wl.nnz4},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
