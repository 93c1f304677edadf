"""GPU parity of the vertex <-> centroid round trip (Sec. 3.2.1, Eq. 2 and Eq. 3) against the
oracle: centroids bit-exact, the P1 integral and the per-iteration errors and fields within
the FP64 tolerance, and a CUDA-graph replay identical to launching the iteration directly.
Every call goes through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2510_18838_gb300 import workloads as W
from tests._helpers import need_gpu, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    need_gpu()
    from paper_2510_18838_gb300 import build, roundtrip
    build.build()
    return roundtrip


def _mesh(n, seed):
    xy, tri = W.jittered_grid_mesh(n, 0.3, seed)
    return np.stack([1.8 + 1.4 * xy[0], -0.8 + 1.6 * xy[1]]), tri


def test_centroids_and_integral(R):
    import torch
    from paper_2510_18838_gb300 import pcms
    xy, tri = _mesh(37, 3)
    m = pcms.Mesh(torch.from_numpy(xy).cuda(), torch.from_numpy(tri).cuda())
    c = m.centroids().cpu().numpy()
    assert np.array_equal(c, oracle.centroids(xy, tri))
    rng = np.random.default_rng(4)
    for f in (np.ones(xy.shape[1]), 2.0 + xy[0] - 3 * xy[1], rng.normal(size=xy.shape[1])):
        g = m.integrate(torch.from_numpy(f).cuda())
        o = oracle.p1_integral(xy, tri, f)
        assert abs(g - o) <= 1e-13 * max(1.0, abs(o))
    assert m.integrate(torch.ones(xy.shape[1], dtype=torch.float64).cuda()) == \
        pytest.approx(1.4 * 1.6, rel=1e-14)
    m.destroy()


@pytest.mark.parametrize("degree", [1, 2])
def test_round_trip_matches_oracle(R, degree):
    n = 40
    xy, tri = _mesh(n, 7)
    f = R.sincos_plus_two(xy)
    r = 2.5 * 1.6 / n
    g = R.run(xy, tri, f, degree, r, weight="c4", iterations=5)
    o = oracle.round_trip(xy, tri, f, degree, r, weight="c4", iterations=5)
    assert normwise_err(g["field"][None], o["fields"][-1][None], np.ones(len(f), bool)) <= 1e-11
    for key in ("accuracy_l2", "accuracy_linf", "conservation"):
        np.testing.assert_allclose(g[key], o[key], rtol=1e-6, atol=1e-12)
    assert g["integral_star"] == pytest.approx(o["integral_star"], rel=1e-13)


def test_graph_replay_equals_direct_launches(R):
    n = 48
    xy, tri = _mesh(n, 8)
    f = R.sincos_plus_two(xy)
    r = 3.0 * 1.6 / n
    a = R.RoundTrip(xy, tri, 2, r)
    a.load(f)
    a.iterate(7)
    direct = a.fv.cpu().numpy()
    a.load(f)
    a.replay(7)
    assert np.array_equal(a.fv.cpu().numpy(), direct)
    a.destroy()


def test_linear_field_survives_many_iterations(R):
    """Reproduction makes a linear field a fixed point: after 50 graph replays it is
    unchanged to rounding, and so is its integral."""
    n = 32
    xy, tri = _mesh(n, 9)
    f = 2.0 + 0.5 * xy[0] - 1.5 * xy[1]
    g = R.run(xy, tri, f, 1, 2.5 * 1.6 / n, iterations=50)
    assert g["accuracy_linf"].max() <= 1e-12
    assert g["conservation"].max() <= 1e-12
