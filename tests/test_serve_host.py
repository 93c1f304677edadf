"""Host-side logic of the serving workload (no GPU): the request stream's statistics and the
operator-cache keys."""
import math

import numpy as np

from paper_2510_18838_gb300 import workloads as W


def test_request_stream_shape():
    reqs = W.request_stream(n_req=2000, seed=501)
    assert len(reqs) == 2000
    arr = np.array([r.arrival_s for r in reqs])
    assert (np.diff(arr) > 0).all()
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 2000.0) < 0.1 / 2000.0          # Poisson rate 2000/s
    kinds = np.array([r.kind for r in reqs])
    assert 0.45 < (kinds == "mesh").mean() < 0.55
    mls = [r for r in reqs if r.kind == "mls"]
    reuse = np.mean([r.reuse_of >= 0 for r in mls])
    assert 0.2 < reuse < 0.4
    fresh = [r for r in mls if r.reuse_of < 0]
    assert 0.4 < np.mean([r.dim == 2 for r in fresh]) < 0.6
    assert 0.4 < np.mean([r.degree == 2 for r in fresh]) < 0.6
    nt = np.array([r.n_tgt for r in reqs])
    assert nt.min() >= 1000 and nt.max() <= 2_000_000
    # log-uniform: the median is near the geometric mean of the range
    assert abs(math.log(np.median(nt)) - 0.5 * (math.log(1e3) + math.log(2e6))) < 0.5
    assert all(1 <= r.n_fields <= 16 for r in reqs)
    # the radius gives 10..300 expected neighbours
    for r in fresh:
        m = math.comb(r.dim + r.degree, r.degree)
        c = math.pi if r.dim == 2 else 4 * math.pi / 3
        k = c * r.n_src * r.radius ** r.dim
        assert max(10, 2 * m) * 0.999 <= k <= 300 * 1.001


def test_reuse_points_to_an_earlier_mls_request_with_the_same_geometry():
    reqs = W.request_stream(n_req=300, seed=9)
    by = {r.rid: r for r in reqs}
    for r in reqs:
        if r.kind == "mls" and r.reuse_of >= 0:
            b = by[r.reuse_of]
            assert b.rid < r.rid and b.kind == "mls" and b.reuse_of < 0   # the root request
            assert (b.dim, b.degree, b.radius, b.n_src, b.n_tgt, b.seed) == \
                   (r.dim, r.degree, r.radius, r.n_src, r.n_tgt, r.seed)


def test_max_pts_caps_sizes():
    reqs = W.request_stream(n_req=200, seed=3, max_pts=5000)
    assert max(r.n_tgt for r in reqs) <= 5000
    assert max(r.n_src for r in reqs if r.kind == "mls") <= 5000
