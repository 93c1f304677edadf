"""GPU parity of the MLS transfer (Sec. 3.2.1) against the FP64 CPU oracle.

Neighbour lists and radius doublings are compared bit-exactly; values norm-wise per
field: <= 1e-12 for the FP64 path and <= 2e-5 for the mixed path; per-target statuses
must be identical. Every call goes through the C ABI (paper_2510_18838_gb300.pcms).
"""
import numpy as np
import pytest

import oracle
from paper_2510_18838_gb300 import workloads as W
from tests._helpers import TOL_FP64, TOL_MIXED, need_gpu, normwise_err, rows_as_sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    need_gpu()
    from paper_2510_18838_gb300 import build, pcms
    build.build()
    return pcms


def cu(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def _case(dim, ns, nt, seed, outside=0.0):
    src = W.uniform_points(ns, dim, seed)
    tgt = W.uniform_points(nt, dim, seed + 1, lo=-outside, hi=1.0 + outside)
    return src, tgt


# ------------------------------------------------------------------ neighbour lists
@pytest.mark.parametrize("dim,prec,min_nb", [(2, "fp64", 0), (2, "mixed", 0), (3, "fp64", 0),
                                              (3, "mixed", 0), (2, "mixed", 12), (3, "fp64", 15),
                                              (3, "mixed", 15)])
def test_neighbor_lists_bit_exact(P, dim, prec, min_nb):
    ns, nt, r = (6000, 1700, 0.03) if dim == 2 else (20000, 1300, 0.06)
    src, tgt = _case(dim, ns, nt, 100 + dim, outside=0.05)
    m = P.create_map(cu(src), cu(tgt), 1, r, precision=prec, min_neighbors=min_nb)
    off, cols, vals, st, kx = (host(x) for x in m.export())
    o_off, o_cols, o_kx = oracle.neighbors(src, tgt, r, min_neighbors=min_nb, degree=1)
    assert np.array_equal(kx, o_kx)
    assert np.array_equal(np.diff(off), np.diff(o_off))
    for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o_off, o_cols)):
        assert np.array_equal(a, b)
    m.destroy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_neighbor_selection_exact_at_the_radius(P, prec):
    """Sources exactly at distance r (dyadic) are excluded; one ulp inside is included."""
    r = 5.0 / 128          # a 3-4-5 triangle with dyadic legs: 3/128, 4/128
    g = (np.arange(8) + 0.5) / 8.0
    tx, ty = np.meshgrid(g, g)
    tgt = np.stack([tx.ravel(), ty.ravel()])
    a, b = 3.0 / 128, 4.0 / 128
    on = [(r, 0.0), (-r, 0.0), (0.0, r), (0.0, -r), (a, b)]      # exactly at distance r
    src = [tgt + np.array(o)[:, None] for o in on]
    for o, ax in [((r, 0.0), 0), ((0.0, -r), 1), ((a, b), 1)]:  # one ulp inside
        p = tgt + np.array(o)[:, None]
        p[ax] = np.nextafter(p[ax], tgt[ax])
        src.append(p)
    src = np.concatenate(src, axis=1)
    m = P.create_map(cu(src), cu(tgt), 0, r, precision=prec)
    off, cols, *_ = (host(x) for x in m.export())
    o_off, o_cols, _ = oracle.neighbors(src, tgt, r, degree=0)
    for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o_off, o_cols)):
        assert np.array_equal(a, b)
    nt = tgt.shape[1]
    exact = set(range(5 * nt))        # the five sources per target at exactly distance r
    assert not exact.intersection(np.asarray(cols).tolist())
    assert all(2 <= len(x) <= 3 for x in rows_as_sets(off, cols))


# ------------------------------------------------------------------ FP64 operator + values
@pytest.mark.parametrize("dim,deg", [(2, 0), (2, 1), (2, 2), (3, 1), (3, 2)])
def test_fp64_map_values_and_shape(P, dim, deg):
    ns, nt, r = (5000, 1500, 0.05) if dim == 2 else (12000, 900, 0.12)
    src, tgt = _case(dim, ns, nt, 200 + 10 * dim + deg)
    f = np.stack([np.sin(3 * src[0]) * np.cos(2 * src[1]), src[0] ** 2 - src[1]])
    m = P.create_map(cu(src), cu(tgt), deg, r)
    out = host(m.apply(cu(f)))
    o = oracle.mls(src, tgt, f, deg, r, shape=True)
    off, cols, vals, st, kx = (host(x) for x in m.export())
    assert np.array_equal(st, o["status"])
    ok = o["status"] == 0
    assert ok.mean() > 0.9
    assert normwise_err(out, o["values"], ok) <= TOL_FP64
    assert np.isnan(out[:, ~ok]).all()
    # shape functions, row by row (compare sorted by column)
    err = 0.0
    scale = np.abs(o["shape"]).max()
    for i in np.nonzero(ok)[0]:
        a = slice(off[i], off[i + 1])
        b = slice(o["offsets"][i], o["offsets"][i + 1])
        ia, ib = np.argsort(cols[a]), np.argsort(o["cols"][b])
        assert np.array_equal(cols[a][ia], o["cols"][b][ib])
        err = max(err, np.abs(vals[a][ia] - o["shape"][b][ib]).max())
    assert err / scale <= TOL_FP64


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 2)])
def test_fp64_one_shot_transfer(P, dim, deg):
    ns, nt, r = (5000, 1500, 0.05) if dim == 2 else (12000, 900, 0.12)
    src, tgt = _case(dim, ns, nt, 300 + 10 * dim + deg)
    f = np.cos(4 * src[0]) + src[1] * src[dim - 1]
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f), deg, r)
    o = oracle.mls(src, tgt, f, deg, r)
    assert np.array_equal(host(st), o["status"])
    ok = o["status"] == 0
    assert normwise_err(host(out), o["values"], ok) <= TOL_FP64


def test_fp64_small_config_full(P):
    """10,000 -> 10,000 uniform 2D, linear basis, Wendland C2, r = 0.03."""
    c = W.mls_2d_small()
    o = oracle.mls(c.src, c.tgt, c.fields, c.degree, c.radius)
    out, st = P.mls_transfer(cu(c.src), cu(c.tgt), cu(c.fields), c.degree, c.radius)
    assert np.array_equal(host(st), o["status"])
    ok = o["status"] == 0
    assert normwise_err(host(out), o["values"], ok) <= TOL_FP64
    m = P.create_map(cu(c.src), cu(c.tgt), c.degree, c.radius)
    out2 = host(m.apply(cu(c.fields)))
    assert normwise_err(out2, o["values"], ok) <= TOL_FP64


@pytest.mark.parametrize("weight", ["wendland_c2", "gaussian", "c4", "const", "noop", "mq", "imq",
                                    "tps", "cubic"])
def test_fp64_every_weight(P, weight):
    src, tgt = _case(2, 4000, 700, 400)
    f = np.sin(5 * src[0]) + src[1]
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f), 1, 0.06, weight=weight)
    o = oracle.mls(src, tgt, f, 1, 0.06, weight=weight)
    assert np.array_equal(host(st), o["status"])
    ok = o["status"] == 0
    assert normwise_err(host(out), o["values"], ok) <= TOL_FP64


def test_fp64_tikhonov(P):
    src, tgt = _case(2, 4000, 700, 410)
    f = np.cos(3 * src[0] + src[1])
    for lam in (1e-3, 0.5):
        out, st = P.mls_transfer(cu(src), cu(tgt), cu(f), 2, 0.06, lam=lam)
        o = oracle.mls(src, tgt, f, 2, 0.06, lam=lam)
        assert np.array_equal(host(st), o["status"])
        assert normwise_err(host(out), o["values"], o["status"] == 0) <= TOL_FP64


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_mixed_values(P, dim, deg):
    ns, nt, r = (20000, 3000, 0.03) if dim == 2 else (40000, 2000, 0.08)
    src, tgt = _case(dim, ns, nt, 500 + 10 * dim + deg)
    f32 = (np.sin(2 * np.pi * src[0]) * np.cos(2 * np.pi * src[1])).astype(np.float32)
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f32), deg, r, precision="mixed")
    o = oracle.mls(src, tgt, f32.astype(np.float64), deg, r)
    assert np.array_equal(host(st), o["status"])
    ok = o["status"] == 0
    assert normwise_err(host(out), o["values"], ok) <= TOL_MIXED
    m = P.create_map(cu(src), cu(tgt), deg, r, precision="mixed")
    out2 = host(m.apply(cu(f32)))
    assert normwise_err(out2, o["values"], ok) <= TOL_MIXED


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("weight", ["gaussian", "c4", "const", "noop", "mq", "imq", "tps",
                                    "cubic"])
def test_mixed_map_every_weight(P, dim, weight):
    """Mixed operators with every weight of Table 1 besides Wendland C2 (the walk with the
    weight kind read at run time), 8 lanes per target: lists bit-exact, statuses equal,
    values within the mixed tolerance."""
    ns, nt, r = (6000, 800, 0.05) if dim == 2 else (20000, 600, 0.09)
    src, tgt = _case(dim, ns, nt, 610 + 10 * dim)
    f = np.sin(5 * src[0]) + src[1]
    m = P.create_map(cu(src), cu(tgt), 1, r, precision="mixed", weight=weight)
    out = host(m.apply(cu(f.astype(np.float32))))
    off, cols, _, st, _ = (host(x) for x in m.export())
    o = oracle.mls(src, tgt, f, 1, r, weight=weight, shape=True)
    assert np.array_equal(st, o["status"])
    for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o["offsets"], o["cols"])):
        assert np.array_equal(a, b)
    ok = o["status"] == 0
    assert ok.mean() > 0.9
    assert normwise_err(out, o["values"], ok) <= TOL_MIXED
    m.destroy()


def test_mixed_multifield_apply_3d(P):
    src = W.slab_points(60000, seed=401)
    tgt = W.uniform_points(3000, 3, 402)
    f = W.trig_fields(src, 16)
    m = P.create_map(cu(src), cu(tgt), 2, 0.07, precision="mixed")
    out = host(m.apply(cu(f)))
    o = oracle.mls(src, tgt, f.astype(np.float64), 2, 0.07)
    ok = o["status"] == 0
    assert ok.mean() > 0.95
    assert normwise_err(out, o["values"], ok) <= TOL_MIXED
    # 1..16 fields give the same numbers as 16 at once
    for nf in (1, 3, 5, 9):
        part = host(m.apply(cu(np.ascontiguousarray(f[:nf]))))
        np.testing.assert_allclose(part[:, ok], out[:nf, ok], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("dim,prec", [(2, "mixed"), (3, "mixed"), (2, "fp64"), (3, "fp64")])
def test_map_rows_longer_than_the_stage(P, dim, prec):
    """Sparse sources plus one dense cluster: the mean neighbour count picks 8 lanes per
    target, while the targets at the cluster see thousands of sources, more than a group
    stages during its walk (384 columns). Their rows are reserved after the walk and walked
    a second time. Lists bit-exact, statuses equal, values within the path's tolerance, and
    the second walk must have run."""
    rng = np.random.default_rng(730 + dim)
    n_bg, n_cl, r = (20000, 2500, 0.02) if dim == 2 else (30000, 3000, 0.07)
    bg = W.uniform_points(n_bg, dim, 731 + dim)
    cl = 0.5 + 0.02 * (rng.random((dim, n_cl)) - 0.5)   # a cube of side 0.02 at the centre
    src = np.ascontiguousarray(np.concatenate([bg, cl], axis=1))
    tgt = np.ascontiguousarray(np.concatenate(
        [W.uniform_points(1500, dim, 733 + dim), 0.5 + 0.06 * (rng.random((dim, 300)) - 0.5)],
        axis=1))
    f = np.sin(2 * np.pi * src[0]) * np.cos(2 * np.pi * src[1])
    P.trace_enable(True, count_only=True)
    m = P.create_map(cu(src), cu(tgt), 2, r, precision=prec)
    out = host(m.apply(cu(f.astype(np.float32) if prec == "mixed" else f)))
    P.trace_enable(False)
    walked_again = P.trace_read().get("count:mls_map_rows_walked_again", (0, 0.0))[0]
    off, cols, _, st, _ = (host(x) for x in m.export())
    o = oracle.mls(src, tgt, f, 2, r, shape=True)
    assert walked_again > 0
    assert np.diff(off).max() > 384
    assert np.array_equal(st, o["status"])
    for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o["offsets"], o["cols"])):
        assert np.array_equal(a, b)
    ok = o["status"] == 0
    assert ok.mean() > 0.95
    assert normwise_err(out, o["values"], ok) <= (TOL_MIXED if prec == "mixed" else TOL_FP64)
    m.destroy()


@pytest.mark.parametrize("dim,nf", [(3, 16), (3, 5), (2, 1), (2, 13)])
def test_tensor_core_apply_matches_the_oracle_and_the_fp32_apply(P, dim, nf):
    """pcms_apply_map_bf16 (BF16 three-term splits on mma.sync, FP32 accumulation) against the
    oracle within the mixed tolerance (the FP32 CUDA-core apply of the same map too, and the
    two against each other); targets outside the box (NaN) stay NaN; a ragged last tile of 16
    targets and rows of uneven length (the dense slab) included."""
    if dim == 3:
        src = W.slab_points(60000, seed=401)
        tgt = W.uniform_points(3001, 3, 402, lo=-0.05, hi=1.05)
        r = 0.07
    else:
        src = W.gaussian_mixture_points(40000, 301, 302)
        tgt = W.uniform_points(2999, 2, 303)
        r = 0.02
    f = W.trig_fields(src, nf)
    m = P.create_map(cu(src), cu(tgt), 2, r, precision="mixed", min_neighbors=10)
    ref = host(m.apply(cu(f)))
    out = host(m.apply_bf16(cu(f)))
    o = oracle.mls(src, tgt, f.astype(np.float64), 2, r, min_neighbors=10, mode="grid")
    ok = o["status"] == 0
    assert np.array_equal(np.isfinite(out).all(axis=0), ok)
    e_tc, e_32 = normwise_err(out, o["values"], ok), normwise_err(ref, o["values"], ok)
    assert e_32 <= TOL_MIXED, e_32
    assert e_tc <= TOL_MIXED, (e_tc, e_32)
    # both are FP32-level results; on rows with a large sum_j |N_j| (far targets of the
    # mixture, whose radius grew) they differ by up to about that sum times 2^-23
    assert normwise_err(out, ref, ok) <= TOL_MIXED
    m.destroy()


def test_mixed_growth_gaussian_mixture(P):
    src = W.gaussian_mixture_points(60000, 301, 302)
    tgt = W.uniform_points(3000, 2, 303)
    f32 = W.sincos_field(src).astype(np.float32)
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f32), 2, 0.01, precision="mixed",
                             min_neighbors=10)
    o = oracle.mls(src, tgt, f32.astype(np.float64), 2, 0.01, min_neighbors=10, mode="grid")
    assert np.array_equal(host(st), o["status"])
    assert normwise_err(host(out), o["values"], o["status"] == 0) <= TOL_MIXED
    m = P.create_map(cu(src), cu(tgt), 2, 0.01, precision="mixed", min_neighbors=10)
    *_, kx = (host(x) for x in m.export())
    assert np.array_equal(kx, o["kexp"])
    assert kx.max() >= 1


@pytest.mark.parametrize("dim,deg,nf,n_src,r", [(3, 2, 5, 40000, 0.09), (2, 2, 16, 60000, 0.03),
                                               (2, 1, 3, 30000, 0.016), (3, 1, 9, 30000, 0.08),
                                               (2, 2, 4, 300000, 0.02)])
def test_mixed_many_field_transfer_applies_rows_as_evaluated(P, dim, deg, nf, n_src, r):
    """Three or more mixed fields: one walk, each operator row applied to all fields as it is
    evaluated (8 and 32 lanes per target, 4 to 16 padded fields). Values against the oracle,
    statuses equal, and the same numbers as the stored operator's apply."""
    src = W.uniform_points(n_src, dim, 51 + nf)
    tgt = W.uniform_points(6000, dim, 52 + nf)
    f = W.trig_fields(src, n_fields=nf, max_deg=2, seed0=60 + nf).astype(np.float32)
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f), deg, r, precision="mixed")
    o = oracle.mls(src, tgt, f.astype(np.float64), deg, r, mode="grid")
    assert np.array_equal(host(st), o["status"])
    ok = o["status"] == 0
    assert normwise_err(host(out), o["values"], ok) <= TOL_MIXED
    m = P.create_map(cu(src), cu(tgt), deg, r, precision="mixed")
    ref = host(m.apply(cu(f)))
    m.destroy()
    np.testing.assert_allclose(host(out)[:, ok], ref[:, ok], rtol=1e-5, atol=1e-5)
    assert np.isnan(host(out)[:, ~ok]).all()


def test_mixed_dense_targets_in_an_estimated_basis(P):
    """The blocked-compensation plan (mean count ~1250): one-sided targets (grown radii at the
    edge of a cluster, the domain boundary) are assembled in tier 1 in a re-centred basis
    estimated from the source cells. Values, statuses and doublings against the oracle, for
    the one-shot transfer and the operator; the estimate takes the place of most tier-2
    walks."""
    src = W.gaussian_mixture_points(400_000, 301, 302)
    tgt = W.uniform_points(3000, 2, 303)
    r = 0.01 * np.sqrt(10.0)
    f32 = W.sincos_field(src).astype(np.float32)
    o = oracle.mls(src, tgt, f32.astype(np.float64), 2, r, min_neighbors=10, mode="grid")
    ok = o["status"] == 0
    P.trace_enable(True, count_only=True)
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f32), 2, r, precision="mixed",
                             min_neighbors=10)
    tr = P.trace_read()
    P.trace_enable(False)
    assert np.array_equal(host(st), o["status"])
    assert normwise_err(host(out), o["values"], ok) <= TOL_MIXED
    n_rc = tr.get("count:mls_tier1_recentred_solves", (0, 0))[0]
    pairs_t2 = tr.get("count:mls_fused_tier2_pairs", (0, 0))[0]
    m = P.create_map(cu(src), cu(tgt), 2, r, precision="mixed", min_neighbors=10)
    offs, *_, kx = (host(x) for x in m.export())
    assert np.array_equal(kx, o["kexp"])
    # without the estimate, tier 2 re-walked the one-sided targets: about 29% of all pairs
    assert n_rc >= 50 and pairs_t2 <= 0.05 * int(offs[-1]), (n_rc, pairs_t2, int(offs[-1]))
    v = host(m.apply(cu(f32[None]))).reshape(o["values"].shape)
    assert normwise_err(v, o["values"], ok) <= TOL_MIXED
    m.destroy()


@pytest.mark.parametrize("dim,prec,deg", [(2, "fp64", 1), (2, "mixed", 2), (3, "mixed", 1),
                                          (3, "fp64", 2)])
def test_global_growth_matches_oracle(P, dim, prec, deg):
    """Global reading of the minimum-count rule: one shared radius r 2^K for every target.
    Neighbour lists, doublings (K everywhere), values and statuses against the oracle's
    global mode, through the operator, the one-shot transfer and the count entry point."""
    ns, nt, r, need = (5000, 1500, 0.01, 12) if dim == 2 else (12000, 900, 0.03, 20)
    src, tgt = _case(dim, ns, nt, 700 + dim, outside=0.25)
    f = np.sin(3 * src[0]) + src[1] * src[-1]
    o = oracle.mls(src, tgt, f, deg, r, min_neighbors=need, mode="grid", growth="global",
                   shape=True)
    K = int(o["kexp"][0])
    assert K >= 2 and (o["kexp"] == K).all()
    dt = np.float64 if prec == "fp64" else np.float32
    tol = TOL_FP64 if prec == "fp64" else TOL_MIXED
    m = P.create_map(cu(src), cu(tgt), deg, r, precision=prec, min_neighbors=need,
                     growth="global")
    off, cols, vals, st, kx = (host(x) for x in m.export())
    assert (kx == K).all() and m.info()["max_radius_doublings"] == K
    assert np.array_equal(st, o["status"])
    for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o["offsets"], o["cols"])):
        assert np.array_equal(a, b)
    ok = o["status"] == 0
    out = host(m.apply(cu(f.astype(dt))))
    assert normwise_err(out[None], o["values"], ok) <= tol
    v, st2 = P.mls_transfer(cu(src), cu(tgt), cu(f.astype(dt)), deg, r, precision=prec,
                            min_neighbors=need, growth="global")
    assert np.array_equal(host(st2), o["status"])
    assert normwise_err(host(v), o["values"], ok) <= tol
    c, k = P.count_neighbors(cu(src), cu(tgt), r, degree=deg, precision=prec,
                             min_neighbors=need, with_doublings=True, growth="global")
    assert np.array_equal(host(c), np.diff(o["offsets"])) and (host(k) == K).all()
    m.destroy()


# ------------------------------------------------------------------ statuses and edge cases
def test_strict_mode_reports_underdetermined(P):
    src, tgt = _case(2, 300, 200, 600, outside=0.5)
    m = P.create_map(cu(src), cu(tgt), 2, 0.05)
    assert m.status_code == P.UNDERDETERMINED
    *_, st, _ = (host(x) for x in m.export())
    o = oracle.mls(src, tgt, np.ones(300), 2, 0.05)
    assert np.array_equal(st, o["status"])
    assert m.info()["n_underdetermined"] == int((o["status"] == 1).sum()) > 0
    out = host(m.apply(cu(np.ones((1, 300)))))
    assert np.isnan(out[0, o["status"] != 0]).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_collinear_neighbours_are_ill_conditioned(P, prec):
    x = np.linspace(0.45, 0.55, 201)
    line = np.stack([x, 0.5 + 0.25 * (x - 0.5)])
    cloud = W.uniform_points(2000, 2, 601)
    cloud = cloud[:, np.hypot(cloud[0] - 0.5, cloud[1] - 0.5) > 0.02]
    src = np.concatenate([line, cloud], axis=1)
    tgt = np.array([[0.5, 0.3], [0.5, 0.3]])
    f = np.ones(src.shape[1])
    dt = np.float64 if prec == "fp64" else np.float32
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f.astype(dt)), 1, 0.004, precision=prec)
    o = oracle.mls(src, tgt, f, 1, 0.004)
    assert o["status"][0] == 2
    assert np.array_equal(host(st), o["status"])
    assert np.isnan(host(out)[0, 0])


def test_empty_and_tiny_inputs(P):
    import torch
    src, tgt = _case(2, 100, 10, 700)
    out, st = P.mls_transfer(cu(src), cu(tgt[:, :0]), cu(np.ones(100)), 1, 0.1)
    assert out.shape == (1, 0)
    out, st = P.mls_transfer(cu(src[:, :0]), cu(tgt), cu(np.ones(0)), 1, 0.1)
    assert (host(st) == 1).all() and np.isnan(host(out)).all()
    m = P.create_map(cu(src), cu(tgt[:, :1]), 0, 0.3)
    assert m.info()["n_tgt"] == 1
    o = oracle.mls(src, tgt[:, :1], np.arange(100.0), 0, 0.3)
    assert normwise_err(host(m.apply(cu(np.arange(100.0)))), o["values"]) <= TOL_FP64


def test_nonfinite_coordinates_rejected(P):
    src, tgt = _case(2, 100, 10, 710)
    src[0, 5] = np.nan
    with pytest.raises(P.PcmsError) as e:
        P.create_map(cu(src), cu(tgt), 1, 0.1)
    assert e.value.status == P.INVALID_ARG


def test_ragged_tile_sizes(P):
    """Target counts that are not multiples of any tile (1, 31, 33, 257, 1031)."""
    src = W.uniform_points(3000, 2, 720)
    for nt in (1, 31, 33, 257, 1031):
        tgt = W.uniform_points(nt, 2, 721 + nt)
        out, st = P.mls_transfer(cu(src), cu(tgt), cu(src[0].copy()), 1, 0.05)
        o = oracle.mls(src, tgt, src[0], 1, 0.05)
        assert np.array_equal(host(st), o["status"])
        assert normwise_err(host(out), o["values"], o["status"] == 0) <= TOL_FP64


# ------------------------------------------------------------------ full-size, sampled
def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


def test_full_size_mls2d_gaussian_mixture_sampled(P):
    """4M Gaussian-mixture sources -> 4M targets, quadratic, r = 0.01, min 10 neighbours,
    mixed precision one-shot transfer: a seeded sample of targets against the oracle."""
    c = W.mls_2d_gaussian()
    f32 = c.fields.astype(np.float32)
    out, st = P.mls_transfer(cu(c.src), cu(c.tgt), cu(f32), c.degree, c.radius,
                             precision="mixed", min_neighbors=c.min_neighbors)
    out, st = host(out), host(st)
    idx = _sample(c.tgt.shape[1], 400, 31)
    o = oracle.mls(c.src, c.tgt[:, idx], f32.astype(np.float64), c.degree, c.radius,
                   min_neighbors=c.min_neighbors, mode="grid")
    assert np.array_equal(st[idx], o["status"])
    assert normwise_err(out[:, idx], o["values"], o["status"] == 0) <= TOL_MIXED
    assert (st == 0).all()


def test_full_size_mls3d_sixteen_fields_sampled(P):
    """8M slab sources -> 8M targets, quadratic, r = 0.012, 16 fields: operator + apply."""
    c = W.mls_3d_slab()
    m = P.create_map(cu(c.src), cu(c.tgt), c.degree, c.radius, precision="mixed")
    out = host(m.apply(cu(c.fields)))
    *_, st, _ = (host(x) for x in m.export())
    idx = _sample(c.tgt.shape[1], 2000, 32)
    o = oracle.mls(c.src, c.tgt[:, idx], c.fields.astype(np.float64), c.degree, c.radius,
                   mode="grid")
    assert np.array_equal(st[idx], o["status"])
    assert normwise_err(out[:, idx], o["values"], o["status"] == 0) <= TOL_MIXED
    # neighbour lists of the sampled targets, bit-exact
    off, cols, *_ = (host(x) for x in m.export())
    o_off, o_cols, _ = oracle.neighbors(c.src, c.tgt[:, idx], c.radius, degree=2, mode="grid")
    for k, i in enumerate(idx):
        assert np.array_equal(np.sort(cols[off[i]:off[i + 1]]), o_cols[o_off[k]:o_off[k + 1]])
    m.destroy()


# ------------------------------------------------------------------ four and five dimensions
def _case_nd(dim, ns, nt, seed):
    src = W.uniform_points(ns, dim, seed)
    tgt = W.uniform_points(nt, dim, seed + 1, lo=0.05, hi=0.95)
    return src, tgt


@pytest.mark.parametrize("dim,deg,min_nb", [(4, 1, 0), (4, 2, 0), (5, 1, 0), (5, 2, 0),
                                            (5, 2, 40), (4, 0, 25)])
def test_nd_map_matches_oracle(P, dim, deg, min_nb):
    """4D/5D (FP64): neighbour lists and doublings bit-exact, statuses identical, operator
    applied to three fields within 1e-12 of the oracle's fit."""
    ns, nt, r = (6000, 700, 0.32) if dim == 4 else (8000, 500, 0.42)
    if min_nb:
        r *= 0.5
    src, tgt = _case_nd(dim, ns, nt, 900 + 10 * dim + deg)
    f = np.stack([np.cos(3 * src[0]) + src[1] * src[dim - 1],
                  src[2] ** 2 - src[3],
                  np.exp(-src[dim - 1]) * src[0]])
    o = oracle.mls(src, tgt, f, deg, r, min_neighbors=min_nb, shape=True)
    m = P.create_map(cu(src), cu(tgt), deg, r, min_neighbors=min_nb)
    off, cols, vals, st, kx = (host(x) for x in m.export())
    assert np.array_equal(kx, o["kexp"])
    assert np.array_equal(st, o["status"])
    for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o["offsets"], o["cols"])):
        assert np.array_equal(a, b)
    ok = o["status"] == 0
    assert ok.mean() > 0.9
    out = host(m.apply(cu(f)))
    assert normwise_err(out, o["values"], ok) <= TOL_FP64
    if min_nb:
        assert kx.max() >= 1
    m.destroy()


@pytest.mark.parametrize("weight", ["wendland_c2", "tps"])
def test_nd_selection_exact_at_the_radius(P, weight):
    """5D: sources exactly at distance r (dyadic offsets along an axis and along
    (1, 2, 2, 4, 0)/32, |.| = 5/32 = r) are excluded; one ulp inside, and inside by 2^-21
    and 2^-19 of r (around the FP32 screen's accept bound), are included; among uniform
    background sources. Both walks (counts and columns) against the oracle's brute force."""
    r = 5.0 / 32
    g = np.array([0.25, 0.75])
    tgt = np.stack(np.meshgrid(*([g] * 5), indexing="ij")).reshape(5, -1)   # 32 dyadic targets
    offs = []
    for d in range(5):
        for sgn in (1.0, -1.0):
            e = np.zeros(5)
            e[d] = sgn * r
            offs.append(e)                                   # exactly at r
    offs.append(np.array([1.0, 2.0, 2.0, 4.0, 0.0]) / 32)    # exactly at r, off the axes
    src = [tgt + o[:, None] for o in offs]
    for d, f in [(0, None), (3, None), (1, 1 - 2.0 ** -21), (4, 1 - 2.0 ** -19)]:
        p = tgt.copy()
        if f is None:                                        # one ulp inside
            p[d] = np.nextafter(tgt[d] + r, tgt[d])
        else:
            p[d] = tgt[d] - r * f
        src.append(p)
    src.append(W.uniform_points(3000, 5, 991))
    src = np.ascontiguousarray(np.concatenate(src, axis=1))
    m = P.create_map(cu(src), cu(tgt), 0, r, weight=weight)
    off, cols, *_ = (host(x) for x in m.export())
    o_off, o_cols, _ = oracle.neighbors(src, tgt, r, weight=weight, degree=0)
    for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o_off, o_cols)):
        assert np.array_equal(a, b)
    nt = tgt.shape[1]
    exact = set(range(11 * nt))                              # the sources at exactly r
    assert not exact.intersection(np.asarray(cols).tolist())
    inside = [set(range((11 + k) * nt, (12 + k) * nt)) for k in range(4)]
    got = set(np.asarray(cols).tolist())
    if weight == "wendland_c2":
        assert all(s <= got for s in inside)
    c = P.count_neighbors(cu(src), cu(tgt), r, degree=0, weight=weight)
    assert np.array_equal(host(c), np.diff(o_off))
    m.destroy()


@pytest.mark.parametrize("dim,weight,lam", [(4, "wendland_c2", 0.0), (5, "c4", 0.0),
                                            (5, "gaussian", 1e-3), (4, "imq", 0.0)])
def test_nd_one_shot_transfer(P, dim, weight, lam):
    ns, nt, r = (5000, 600, 0.35) if dim == 4 else (7000, 400, 0.45)
    src, tgt = _case_nd(dim, ns, nt, 950 + dim)
    f = np.sin(2 * src[0]) * np.cos(src[1]) + src[dim - 1]
    out, st = P.mls_transfer(cu(src), cu(tgt), cu(f), 2, r, weight=weight, lam=lam)
    o = oracle.mls(src, tgt, f, 2, r, weight=weight, lam=lam)
    assert np.array_equal(host(st), o["status"])
    assert normwise_err(host(out), o["values"], o["status"] == 0) <= TOL_FP64
    c = P.count_neighbors(cu(src), cu(tgt), r, degree=2, weight=weight)
    off, _, _ = oracle.neighbors(src, tgt, r, weight=weight, degree=2)
    assert np.array_equal(host(c), np.diff(off))


def test_nd_global_growth_and_strict_mode(P):
    src, tgt = _case_nd(5, 4000, 300, 977)
    tgt = np.ascontiguousarray(tgt * 1.3 - 0.15)   # some targets outside the sources' box
    f = src[0] + 2 * src[4]
    o = oracle.mls(src, tgt, f, 1, 0.15, min_neighbors=12, growth="global")
    K = int(o["kexp"][0])
    m = P.create_map(cu(src), cu(tgt), 1, 0.15, min_neighbors=12, growth="global")
    *_, st, kx = (host(x) for x in m.export())
    assert (kx == K).all() and K >= 1
    assert np.array_equal(st, o["status"])
    assert normwise_err(host(m.apply(cu(f))), o["values"], o["status"] == 0) <= TOL_FP64
    m.destroy()
    m2 = P.create_map(cu(src), cu(tgt), 2, 0.15)     # user radius: underdetermined targets
    assert m2.status_code == P.UNDERDETERMINED
    m2.destroy()


# ------------------------------------------------------------------ ill-conditioned fits
@pytest.mark.parametrize("dim,prec,form,nf", [(3, "mixed", "oneshot", 1), (3, "mixed", "oneshot", 5),
                                              (3, "mixed", "map", 5), (3, "fp64", "map", 2),
                                              (3, "fp64", "oneshot", 1), (2, "mixed", "map", 3)])
def test_ill_conditioned_fits_match_the_oracle(P, dim, prec, form, nf):
    """Quadratic fits with few neighbours outside and at the edge of the sources' box (one
    radius beyond it): extrapolating and corner targets whose neighbourhoods are nearly
    degenerate, where normal equations lose up to the square of the Vandermonde matrix's
    condition number. Such targets are solved again by Householder QR in FP64, so every
    target stays within the path's tolerance of the oracle (QR by definition), statuses
    included, for one-shot transfers, cached operators and their export."""
    ns, nt, k = (9000, 2500, 14) if dim == 3 else (5000, 2500, 10)
    src = W.uniform_points(ns, dim, 700 + dim)
    tgt = W.uniform_points(nt, dim, 701 + dim, lo=-0.05, hi=1.05)
    ball = np.pi if dim == 2 else 4.0 / 3.0 * np.pi
    r = (k / (ball * ns)) ** (1.0 / dim)
    f = W.trig_fields(src, n_fields=nf, max_deg=2, seed0=705)
    dt = np.float32 if prec == "mixed" else np.float64
    o = oracle.mls(src, tgt, f.astype(np.float64), 2, r, mode="grid")
    tol = TOL_MIXED if prec == "mixed" else TOL_FP64
    if form == "oneshot":
        out, st = P.mls_transfer(cu(src), cu(tgt), cu(f.astype(dt)), 2, r, precision=prec)
        st = host(st)
    else:
        m = P.create_map(cu(src), cu(tgt), 2, r, precision=prec)
        out = m.apply(cu(f.astype(dt)))
        off, cols, vals, st, _ = (host(x) for x in m.export())
        o_off, o_cols, _ = oracle.neighbors(src, tgt, r, mode="grid")
        for a, b in zip(rows_as_sets(off, cols), rows_as_sets(o_off, o_cols)):
            assert np.array_equal(a, b)   # rows replaced by the QR pass keep their sources
        m.destroy()
    assert np.array_equal(st, o["status"])
    ok = o["status"] == 0
    assert (ok.sum() > 0.4 * nt) and (~ok).sum() > 0
    got = host(out)
    assert np.isnan(got[:, ~ok]).all()
    if prec == "mixed":
        assert normwise_err(got, o["values"], ok) <= tol
        return
    # FP64: QR in the oracle and on the GPU are each backward stable, so they agree to about
    # cond(B) 2^-53 per target, B = diag(sqrt(w)) A; beyond cond(B) ~ 1e3 that exceeds 1e-12.
    # Targets up to that condition meet 1e-12; every target meets 64 cond(B) 2^-53.
    o_off, o_cols, _ = oracle.neighbors(src, tgt, r, mode="grid")
    cond = np.ones(nt)
    for i in np.nonzero(ok)[0]:
        js = o_cols[o_off[i]:o_off[i + 1]]
        u = (src[:, js] - tgt[:, i:i + 1]) / r
        q = np.sqrt((u * u).sum(axis=0))
        w = (1 - q) ** 4 * (4 * q + 1)            # Wendland C2
        cols_a = [np.ones_like(q)] + [u[d] for d in range(dim)]
        cols_a += [u[a] * u[b] for a in range(dim) for b in range(a, dim)]
        B = np.sqrt(w)[:, None] * np.stack(cols_a, axis=1)
        sv = np.linalg.svd(B, compute_uv=False)
        cond[i] = sv[0] / sv[-1]
    scale = np.max(np.abs(o["values"][:, ok]), axis=1)
    err = (np.abs(got - o["values"]) / scale[:, None]).max(axis=0)
    well = ok & (cond <= 1e3)
    assert well.sum() > 0.3 * nt
    assert err[well].max() <= TOL_FP64, err[well].max()
    assert (err[ok] <= np.maximum(TOL_FP64, 64 * cond[ok] * 2.0 ** -53)).all()
