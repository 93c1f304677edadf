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


def test_server_requests_are_checked_before_submission():
    """A serving request's tensors are used in place after submit returns, so a wrong dtype,
    shape or layout is refused in the binding instead of being copied or misread."""
    import types

    import pytest
    import torch

    from paper_2510_18838_gb300 import pcms
    fake = types.SimpleNamespace()          # never reached: the checks come first
    src = torch.zeros((2, 10), dtype=torch.float64)
    tgt = torch.zeros((2, 4), dtype=torch.float64)
    f = torch.zeros((3, 10), dtype=torch.float32)
    out = torch.zeros((3, 4), dtype=torch.float32)
    cases = [
        dict(src=src.float()),                                    # coordinates not FP64
        dict(fields=f.double()),                                  # mixed maps take FP32 fields
        dict(out=torch.zeros((3, 5), dtype=torch.float32)),       # wrong target count
        dict(fields=torch.zeros((10, 3), dtype=torch.float32).t()),   # not contiguous
        dict(tgt=torch.zeros((3, 4), dtype=torch.float64)),       # other dimension
    ]
    for c in cases:
        a = dict(src=src, tgt=tgt, fields=f, out=out)
        a.update(c)
        with pytest.raises((TypeError, ValueError)):
            pcms.Server.submit_mls(fake, a["src"], a["tgt"], a["fields"], a["out"], 1, 0.1)
    with pytest.raises(TypeError):
        pcms.Server.submit_mls(fake, src, tgt, f, out, 1, 0.1, precision="fp64")
    xy = torch.zeros((2, 9), dtype=torch.float64)
    tri = torch.zeros((3, 8), dtype=torch.int32)
    pts = torch.zeros((2, 5), dtype=torch.float64)
    elem = torch.zeros(5, dtype=torch.int32)
    with pytest.raises(TypeError):
        pcms.Server.submit_mesh(fake, xy, tri.long(), pts, None, None, elem)
    with pytest.raises(ValueError):
        pcms.Server.submit_mesh(fake, xy, tri, pts, torch.zeros(9, dtype=torch.float64), None,
                                elem)
    with pytest.raises(ValueError):
        pcms.Server.submit_mesh(fake, xy, tri, pts, torch.zeros(8, dtype=torch.float64),
                                torch.zeros(5, dtype=torch.float64), elem)
