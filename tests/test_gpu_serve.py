"""Serving: each request's result is the same alone and in the concurrent mix (within the
stated tolerances), the memory cap is respected, and oversized requests are refused."""
import numpy as np
import pytest

from paper_2510_18838_gb300 import workloads as W
from tests._helpers import TOL_FP64, TOL_MIXED, need_gpu, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    from paper_2510_18838_gb300 import build, pcms, serve
    build.build()
    return torch, pcms, serve


def _alone(pcms, d):
    r, t = d.req, d.tensors
    if r.kind == "mesh":
        mesh = pcms.Mesh(t["xy"], t["tri"])
        e, _, v = mesh.locate_interp(t["pts"], t["field"], with_dim=False)
        return e.cpu().numpy(), v.cpu().numpy()
    if r.n_fields <= 2:
        out, _ = pcms.mls_transfer(t["src"], t["tgt"], t["fields"], r.degree, r.radius,
                                   precision="mixed", with_status=False)
    else:
        m = pcms.create_map(t["src"], t["tgt"], r.degree, r.radius, precision="mixed")
        out = m.apply(t["fields"])
        m.destroy()
    return out.cpu().numpy()


@pytest.mark.parametrize("n_slots", [1, 6])
def test_alone_equals_in_the_mix(env, n_slots):
    torch, pcms, serve = env
    reqs = W.request_stream(n_req=48, seed=77, pts_hi=60000, max_pts=60000)
    assert {r.kind for r in reqs} == {"mls", "mesh"}
    assert any(r.reuse_of >= 0 for r in reqs)
    dreqs = serve.materialize(reqs, torch.device("cuda", 0))
    stats = serve.run_served(dreqs, n_slots=n_slots, mem_cap=4 << 30)
    assert stats["failed"] == 0
    assert stats["peak_bytes"] <= 4 << 30
    for d in dreqs:
        r, t = d.req, d.tensors
        if r.kind == "mesh":
            e_mix, v_mix = t["elem"].cpu().numpy(), t["values"].cpu().numpy()
            e_al, v_al = _alone(pcms, d)
            assert np.array_equal(e_mix, e_al)
            inside = e_al >= 0
            assert normwise_err(v_mix, v_al, inside) <= TOL_FP64
        else:
            mix = t["out"].cpu().numpy()
            al = _alone(pcms, d)
            ok = np.isfinite(al).all(axis=0)
            assert np.array_equal(np.isfinite(mix).all(axis=0), ok)
            assert normwise_err(mix, al, ok) <= TOL_MIXED, r


def test_cache_reuse_and_capacity(env):
    torch, pcms, serve = env
    dev = torch.device("cuda", 0)
    src = torch.rand((2, 20000), dtype=torch.float64, device=dev)
    tgt = torch.rand((2, 5000), dtype=torch.float64, device=dev)
    f1 = torch.rand((3, 20000), dtype=torch.float32, device=dev)
    f2 = torch.rand((5, 20000), dtype=torch.float32, device=dev)
    o1 = torch.empty((3, 5000), dtype=torch.float32, device=dev)
    o2 = torch.empty((5, 5000), dtype=torch.float32, device=dev)
    s = pcms.Server(n_slots=2, mem_cap_bytes=2 << 30)
    s.submit_mls(src, tgt, f1, o1, 2, 0.03, map_key=7)
    s.submit_mls(src, tgt, f2, o2, 2, 0.03, map_key=7, reuse=True)
    s.drain(120)
    res = sorted(s.poll(8), key=lambda x: x["ticket"])
    assert [x["status"] for x in res] == [pcms.OK, pcms.OK]
    assert res[1]["cached"] and not res[0]["cached"]
    assert s.memory()["cached_maps"] == 1
    m = pcms.create_map(src, tgt, 2, 0.03, precision="mixed")
    ref = m.apply(f2).cpu().numpy()
    assert normwise_err(o2.cpu().numpy(), ref) <= TOL_MIXED
    s.close()
    # a request whose estimate exceeds the cap is refused, the server keeps running
    s = pcms.Server(n_slots=1, mem_cap_bytes=1 << 20)
    s.submit_mls(src, tgt, f1, o1, 2, 0.03)
    s.drain(60)
    assert s.poll(4)[0]["status"] == pcms.CAPACITY
    s.close()


def test_reuse_that_does_not_fit_beside_its_operator(env):
    """Eviction must never free the operator that the request being admitted is about to use:
    under a cap that holds the cached operator but not the reuse request's scratch beside it,
    the request drops the operator, builds it again and returns the right values."""
    torch, pcms, serve = env
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(5)
    src = torch.rand((2, 20000), dtype=torch.float64, device=dev, generator=g)
    tgt = torch.rand((2, 5000), dtype=torch.float64, device=dev, generator=g)
    f1 = torch.rand((3, 20000), dtype=torch.float32, device=dev, generator=g)
    f2 = torch.rand((5, 20000), dtype=torch.float32, device=dev, generator=g)
    o1 = torch.empty((3, 5000), dtype=torch.float32, device=dev)
    o2 = torch.empty((5, 5000), dtype=torch.float32, device=dev)
    s = pcms.Server(n_slots=1, mem_cap_bytes=2 << 30)
    s.submit_mls(src, tgt, f1, o1, 2, 0.03, map_key=7)
    s.drain(120)
    op_bytes = s.memory()["in_use"]          # the cached operator alone
    s.close()
    assert op_bytes > 0
    # room for the operator plus 1 MiB: less than the reuse's scratch and fixed 1 MiB slack
    s = pcms.Server(n_slots=1, mem_cap_bytes=op_bytes + (1 << 20))
    s.submit_mls(src, tgt, f1, o1, 2, 0.03, map_key=7, bytes_hint=op_bytes)
    s.drain(120)
    s.submit_mls(src, tgt, f2, o2, 2, 0.03, map_key=7, reuse=True, bytes_hint=op_bytes)
    s.drain(120)
    res = sorted(s.poll(8), key=lambda x: x["ticket"])
    s.close()
    assert [x["status"] for x in res] == [pcms.OK, pcms.OK]
    assert not res[1]["cached"]               # rebuilt, not applied from a freed operator
    m = pcms.create_map(src, tgt, 2, 0.03, precision="mixed")
    assert normwise_err(o2.cpu().numpy(), m.apply(f2).cpu().numpy()) <= TOL_MIXED
    assert normwise_err(o1.cpu().numpy(), m.apply(f1).cpu().numpy()) <= TOL_MIXED
    m.destroy()


def test_a_failing_request_does_not_disturb_the_others(env):
    """A request that fails while running (a non-finite source coordinate, found by the
    library's bounding-box pass) comes back with its error status; requests around it, in
    other slots and after it in the same slot, complete with correct results."""
    torch, pcms, serve = env
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(11)
    src = torch.rand((2, 30000), dtype=torch.float64, device=dev, generator=g)
    tgt = torch.rand((2, 8000), dtype=torch.float64, device=dev, generator=g)
    f = torch.rand((2, 30000), dtype=torch.float32, device=dev, generator=g)
    bad = src.clone()
    bad[0, 1234] = float("nan")
    outs = [torch.empty((2, 8000), dtype=torch.float32, device=dev) for _ in range(5)]
    s = pcms.Server(n_slots=2, mem_cap_bytes=2 << 30)
    tickets = []
    for i in range(5):
        tickets.append(s.submit_mls(bad if i == 2 else src, tgt, f, outs[i], 2, 0.03))
    s.drain(120)
    res = {x["ticket"]: x["status"] for x in s.poll(16)}
    s.close()
    assert res[tickets[2]] == pcms.INVALID_ARG
    ref, _ = pcms.mls_transfer(src, tgt, f, 2, 0.03, precision="mixed", with_status=False)
    ref = ref.cpu().numpy()
    ok = np.isfinite(ref).all(axis=0)
    for i in (0, 1, 3, 4):
        assert res[tickets[i]] == pcms.OK
        assert normwise_err(outs[i].cpu().numpy(), ref, ok) <= TOL_MIXED


@pytest.mark.parametrize("pin", [False, True])
def test_host_io_requests_match_device_requests(env, pin):
    """Requests whose buffers are host memory, ordinary or page-locked (the server stages the
    copies on each slot's stream), give bit-identical results to the same requests on
    device buffers."""
    torch, pcms, serve = env
    reqs = W.request_stream(n_req=40, seed=78, pts_hi=40000, max_pts=40000)
    dreqs = serve.materialize(reqs, torch.device("cuda", 0))
    host = serve.to_host(dreqs, pin=pin)
    assert all(not v.is_cuda for d in host for v in d.tensors.values())
    st_d = serve.run_served(dreqs, n_slots=4, mem_cap=2 << 30)
    st_h = serve.run_served(host, n_slots=4, mem_cap=2 << 30)
    assert st_d["failed"] == 0 and st_h["failed"] == 0
    for d, h in zip(dreqs, host):
        for k in serve.OUTPUT_KEYS:
            if k in d.tensors:
                a, b = d.tensors[k].cpu().numpy(), h.tensors[k].numpy()
                assert np.array_equal(a, b, equal_nan=True), (d.req, k)


def test_fp64_reuse_reserves_the_padded_apply_scratch(env):
    """A float64 request that reuses a cached operator with 9 fields: the apply pads the
    fields to 16 per row for its scratch (the fields in source order and the staged result,
    16 * 8 bytes per source and per target). The server's reservation for the reuse, seen
    in its peak above the cached operator, must cover that, and the values must equal a
    fresh map's."""
    torch, pcms, serve = env
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(21)
    ns, nt, nf = 30000, 12000, 9
    src = torch.rand((2, ns), dtype=torch.float64, device=dev, generator=g)
    tgt = torch.rand((2, nt), dtype=torch.float64, device=dev, generator=g)
    f1 = torch.rand((1, ns), dtype=torch.float64, device=dev, generator=g)
    f9 = torch.rand((nf, ns), dtype=torch.float64, device=dev, generator=g)
    o1 = torch.empty((1, nt), dtype=torch.float64, device=dev)
    o9 = torch.empty((nf, nt), dtype=torch.float64, device=dev)
    s = pcms.Server(n_slots=1, mem_cap_bytes=2 << 30)
    s.submit_mls(src, tgt, f1, o1, 1, 0.03, precision="fp64", map_key=3)
    s.drain(120)
    op_bytes = s.memory()["in_use"]
    s.close()
    s = pcms.Server(n_slots=1, mem_cap_bytes=2 << 30)
    s.submit_mls(src, tgt, f1, o1, 1, 0.03, precision="fp64", map_key=3)
    s.drain(120)
    assert s.memory()["in_use"] == op_bytes
    s.submit_mls(src, tgt, f9, o9, 1, 0.03, precision="fp64", map_key=3, reuse=True)
    s.drain(120)
    res = sorted(s.poll(8), key=lambda x: x["ticket"])
    mem = s.memory()
    s.close()
    assert [x["status"] for x in res] == [pcms.OK, pcms.OK]
    assert res[1]["cached"]
    scratch = (ns + nt) * 16 * 8
    assert mem["peak"] - op_bytes >= scratch, (mem, op_bytes, scratch)
    m = pcms.create_map(src, tgt, 1, 0.03, precision="fp64")
    ref = m.apply(f9).cpu().numpy()
    m.destroy()
    ok = np.isfinite(ref).all(axis=0)
    assert normwise_err(o9.cpu().numpy(), ref, ok) <= TOL_FP64


def _batchable(d, reused):
    r = d.req
    return (r.kind == "mls" and r.reuse_of < 0 and r.rid not in reused
            and r.n_src <= 8192 and r.n_tgt <= 8192)


def test_batched_requests_are_bitwise_the_same_alone_and_match_the_oracle(env):
    """Small one-shot MLS requests go through the batched path (several per graph replay).
    Each one's result is bitwise the result of the same request served alone, and a sample
    of them matches the FP64 oracle within the mixed tolerance."""
    import oracle
    torch, pcms, serve = env
    reqs = W.request_stream(n_req=60, seed=79, pts_hi=50000, max_pts=50000)
    dreqs = serve.materialize(reqs, torch.device("cuda", 0))
    reused = {d.req.reuse_of for d in dreqs if d.req.kind == "mls" and d.req.reuse_of >= 0}
    small = [i for i, d in enumerate(dreqs) if _batchable(d, reused)]
    assert len(small) >= 4
    st = serve.run_served(dreqs, n_slots=6, mem_cap=4 << 30)
    assert st["failed"] == 0
    assert st["batched_requests"] >= len(small) and st["batches"] < st["batched_requests"]
    mix = {i: dreqs[i].tensors["out"].cpu().numpy().copy() for i in small}
    for i in small[:6]:
        one = serve.run_served([dreqs[i]], n_slots=1, mem_cap=4 << 30)
        assert one["failed"] == 0 and one["batched_requests"] == 1
        assert np.array_equal(dreqs[i].tensors["out"].cpu().numpy(), mix[i], equal_nan=True)
    rng = np.random.default_rng(5)
    for i in small[:4]:
        d = dreqs[i]
        t = {k: v.cpu().numpy() for k, v in d.tensors.items()}
        sel = rng.choice(d.req.n_tgt, min(400, d.req.n_tgt), replace=False)
        o = oracle.mls(t["src"], t["tgt"][:, sel], t["fields"].astype(np.float64), d.req.degree,
                       d.req.radius, mode="grid")
        ok = o["status"] == 0
        assert np.array_equal(np.isfinite(mix[i][:, sel]).all(axis=0), ok)
        assert normwise_err(mix[i][:, sel], o["values"], ok) <= TOL_MIXED


def test_batching_off_gives_the_general_path(env):
    """With batching off the same requests run one by one through the general path; the two
    paths agree within the mixed tolerance, target by target status included."""
    torch, pcms, serve = env
    reqs = W.request_stream(n_req=40, seed=80, pts_hi=30000, max_pts=30000)
    dreqs = serve.materialize(reqs, torch.device("cuda", 0))
    a = serve.run_served(dreqs, n_slots=4, mem_cap=4 << 30)
    outs = [d.tensors["out"].cpu().numpy().copy() if d.req.kind == "mls" else None for d in dreqs]
    b = serve.run_served(dreqs, n_slots=4, mem_cap=4 << 30, batch_max=0)
    assert a["failed"] == 0 and b["failed"] == 0
    assert a["batched_requests"] > 0 and b["batched_requests"] == 0
    for d, o in zip(dreqs, outs):
        if o is None:
            continue
        g = d.tensors["out"].cpu().numpy()
        ok = np.isfinite(g).all(axis=0)
        assert np.array_equal(np.isfinite(o).all(axis=0), ok)
        assert normwise_err(o, g, ok) <= TOL_MIXED
