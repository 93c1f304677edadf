"""GPU parity of the batched one-shot MLS transfer (pcms_mls_transfer_batch, Sec. 3.2.1,
Eq. 1) against the FP64 CPU oracle.

Every problem of a batch is compared with the oracle on its own: values norm-wise per field
within the mixed path's 2e-5, per-target statuses identical (OK, underdetermined,
ill-conditioned). The cases cover both lane widths (8 and 32 lanes per target), degrees 0-2
in 2D and 3D, 1 to 16 fields, every weight kind, targets outside the sources' box (one-sided
neighbourhoods, which the FP32 conditioning estimate sends to the FP64 assembly), a
clustered problem whose densest targets overflow the per-target stage (the walk is repeated),
empty problems, and a problem with a non-finite coordinate. A problem's result does not
depend on the rest of its batch (bitwise).
"""
import numpy as np
import pytest

import oracle
from paper_2510_18838_gb300 import workloads as W
from tests._helpers import TOL_MIXED, need_gpu, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    need_gpu()
    from paper_2510_18838_gb300 import build, pcms
    build.build()
    return pcms


def cu(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def problem(dim, ns, nt, seed, k, degree, nf, outside=0.0, weight="wendland_c2", src=None):
    """sources U[0,1]^dim, targets U[-outside, 1+outside]^dim, radius giving k neighbours on
    average, nf random trigonometric fields"""
    if src is None:
        src = W.uniform_points(ns, dim, seed)
    ns = src.shape[1]
    tgt = W.uniform_points(nt, dim, seed + 1, lo=-outside, hi=1.0 + outside)
    ball = np.pi if dim == 2 else 4.0 / 3.0 * np.pi
    r = (k / (ball * ns)) ** (1.0 / dim)
    f = W.trig_fields(src, n_fields=nf, max_deg=2, seed0=seed + 7)
    return dict(src=src, tgt=tgt, fields=f, degree=degree, radius=r, weight=weight)


def to_dev(p):
    import torch
    d = dict(p)
    d["src"] = cu(p["src"], torch.float64)
    d["tgt"] = cu(p["tgt"], torch.float64)
    d["fields"] = cu(p["fields"], torch.float32)
    return d


def check_against_oracle(p, out, st):
    o = oracle.mls(p["src"], p["tgt"], p["fields"].astype(np.float64), p["degree"], p["radius"],
                   weight=p["weight"], mode="grid")
    st = st.cpu().numpy()
    assert np.array_equal(st, o["status"]), (np.bincount(st, minlength=3),
                                              np.bincount(o["status"], minlength=3))
    ok = o["status"] == 0
    got = out.cpu().numpy()
    assert np.isnan(got[:, ~ok]).all()
    assert np.isfinite(got[:, ok]).all()
    err = normwise_err(got, o["values"], ok)
    assert err <= TOL_MIXED, err
    return err


CASES = [
    # dim, ns, nt, seed, k (mean neighbours), degree, fields, outside
    (2, 3000, 1500, 11, 12, 1, 1, 0.0),
    (2, 5000, 1200, 13, 30, 2, 3, 0.05),
    (2, 4000, 900, 15, 200, 2, 16, 0.0),      # 32 lanes per target
    (2, 2000, 700, 17, 8, 0, 2, 0.0),          # Shepard
    (3, 6000, 1100, 19, 40, 1, 4, 0.0),
    (3, 9000, 1000, 21, 70, 2, 16, 0.05),
    (3, 12000, 600, 23, 250, 2, 5, 0.0),       # 32 lanes per target
    (3, 3000, 500, 25, 20, 0, 1, 0.0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}k{c[4]}deg{c[5]}f{c[6]}" for c in CASES])
def test_batch_item_matches_oracle(P, case):
    dim, ns, nt, seed, k, deg, nf, outside = case
    p = problem(dim, ns, nt, seed, k, deg, nf, outside)
    outs, sts, res = P.mls_transfer_batch([to_dev(p)])
    assert res == [P.OK]
    check_against_oracle(p, outs[0], sts[0])


def test_mixed_batch_each_item_matches_oracle_and_is_independent_of_the_batch(P):
    """All the cases above in one batch (several shape classes): each matches the oracle, and
    each result is bitwise the result of the problem submitted alone."""
    ps = [problem(*c) for c in CASES]
    dev = [to_dev(p) for p in ps]
    outs, sts, res = P.mls_transfer_batch(dev)
    assert res == [P.OK] * len(ps)
    for p, o, s in zip(ps, outs, sts):
        check_against_oracle(p, o, s)
    for i in (0, 2, 5, 6):
        o1, s1, r1 = P.mls_transfer_batch([dev[i]])
        assert r1 == [P.OK]
        assert np.array_equal(o1[0].cpu().numpy(), outs[i].cpu().numpy(), equal_nan=True)
        assert np.array_equal(s1[0].cpu().numpy(), sts[i].cpu().numpy())


@pytest.mark.parametrize("weight", ["gaussian", "c4", "const", "noop", "mq", "imq", "tps", "cubic"])
def test_batch_every_weight(P, weight):
    p = problem(2, 3000, 600, 31, 25, 1, 2, 0.0, weight=weight)
    outs, sts, res = P.mls_transfer_batch([to_dev(p)])
    assert res == [P.OK]
    check_against_oracle(p, outs[0], sts[0])


def test_batch_dense_cluster_spills_the_stage(P):
    """Gaussian-mixture sources with a radius that puts several hundred sources in the
    densest targets' balls while the mean stays below 160 (8 lanes, a 256-entry stage): those
    targets walk their rows again for the FP64 moments and the operator rows."""
    src = W.gaussian_mixture_points(6000, seed_centres=41, seed_pts=42)
    p = problem(2, 6000, 1500, 43, 40, 2, 3, 0.0, src=src)
    off, _, _ = oracle.neighbors(p["src"], p["tgt"], p["radius"], mode="grid")
    counts = np.diff(off)
    assert counts.max() > 256 and counts.mean() < 160   # some targets overflow the stage
    outs, sts, res = P.mls_transfer_batch([to_dev(p)])
    assert res == [P.OK]
    check_against_oracle(p, outs[0], sts[0])


def test_batch_degenerate_problems(P):
    """No sources (every target underdetermined), no targets, collinear sources with a
    quadratic basis (ill-conditioned), and a non-finite coordinate (that item alone fails)."""
    import torch
    a = problem(2, 1000, 300, 51, 15, 1, 2)
    empty_src = dict(a, src=np.zeros((2, 0)), fields=np.zeros((2, 0), np.float32))
    no_tgt = dict(a, tgt=np.zeros((2, 0)))
    line = np.stack([np.linspace(0, 1, 800), np.full(800, 0.5)])
    coll = problem(2, 800, 200, 53, 30, 2, 1, src=line)
    coll["tgt"] = np.stack([np.linspace(0.1, 0.9, 200), np.full(200, 0.5)])
    bad = problem(2, 1000, 300, 55, 15, 1, 1)
    bad["src"] = bad["src"].copy()
    bad["src"][1, 17] = np.nan
    items = [empty_src, no_tgt, coll, bad, a]
    outs, sts, res = P.mls_transfer_batch([to_dev(p) for p in items])
    assert res == [P.OK, P.OK, P.OK, P.INVALID_ARG, P.OK]
    assert (sts[0].cpu().numpy() == 1).all() and np.isnan(outs[0].cpu().numpy()).all()
    assert outs[1].shape == (2, 0)
    st = sts[2].cpu().numpy()
    assert (st == 2).all(), np.bincount(st)
    check_against_oracle(coll, outs[2], sts[2])
    check_against_oracle(a, outs[4], sts[4])


def test_batch_rejects_items_beyond_its_limits(P):
    import torch
    p = to_dev(problem(2, 1000, 100, 61, 15, 1, 1))
    big = dict(p, tgt=torch.rand((2, P.BATCH_MAX_POINTS + 1), dtype=torch.float64, device="cuda"))
    with pytest.raises(P.PcmsError):
        P.mls_transfer_batch([p, big])
    with pytest.raises(P.PcmsError):
        P.mls_transfer_batch([dict(p, degree=3)])
