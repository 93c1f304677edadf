"""GPU parity of point localization + barycentric interpolation (Sec. 3.3) against the
oracle: element ids and entity dimensions bit-exact, values within 1e-12."""
import numpy as np
import pytest

import oracle
from paper_2510_18838_gb300 import workloads as W
from tests._helpers import TOL_FP64, need_gpu, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    need_gpu()
    from paper_2510_18838_gb300 import build, pcms
    build.build()
    return pcms


def cu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _check(P, xy, tri, pts, field, mode="exhaustive"):
    mesh = P.Mesh(cu(xy), cu(tri))
    elem, edim, vals = (host(x) for x in mesh.locate_interp(cu(pts), cu(field)))
    o_elem, o_dim, o_vals = oracle.locate(xy, tri, pts, field=field, mode=mode)
    assert np.array_equal(elem, o_elem)
    assert np.array_equal(edim, o_dim)
    inside = o_elem >= 0
    assert np.isnan(vals[~inside]).all()
    assert normwise_err(vals, o_vals, inside) <= TOL_FP64
    mesh.destroy()
    return elem, edim


def test_unjittered_dyadic_edges_and_vertices(P):
    n = 16
    xy, tri = W.jittered_grid_mesh(n, jitter=0.0)
    rng = np.random.default_rng(11)
    pts = np.concatenate([rng.integers(0, 64 * n + 1, size=(2, 3000)) / (64.0 * n),
                          rng.integers(0, n + 1, size=(2, 300)) / float(n),
                          rng.integers(0, 2 * n + 1, size=(2, 300)) / (2.0 * n),
                          np.array([[-0.5, 1.5, 0.25, 1.0], [0.5, 0.5, -1e-300, 1.0]])], axis=1)
    f = xy[0] ** 2 + 3 * xy[0] * xy[1]
    elem, edim = _check(P, xy, tri, pts, f)
    assert (edim == 0).sum() > 100 and (edim == 1).sum() > 100 and (edim == 2).sum() > 1000


def test_jittered_with_vertices_and_edge_points(P):
    xy, tri = W.jittered_grid_mesh(64, 0.3, seed=12)
    pts = W.uniform_points(20000, 2, 13, lo=-0.02, hi=1.02)
    mid = 0.5 * (xy[:, tri[0]] + xy[:, tri[2]])          # on the shared diagonal (up to rounding)
    pts = np.concatenate([pts, xy, mid[:, :2000]], axis=1)
    f = np.sin(3 * xy[0]) + xy[1]
    _check(P, xy, tri, pts, f)


def test_linear_field_exact_and_orientation_independent(P):
    xy, tri = W.jittered_grid_mesh(32, 0.3, seed=14)
    pts = W.uniform_points(20000, 2, 15)
    f = 1.5 - 2.0 * xy[0] + 0.25 * xy[1]
    mesh = P.Mesh(cu(xy), cu(tri))
    _, _, v = mesh.locate_interp(cu(pts), cu(f))
    np.testing.assert_allclose(host(v), 1.5 - 2.0 * pts[0] + 0.25 * pts[1], rtol=0, atol=1e-13)
    # clockwise copies of every triangle: same ids, same classification
    tri_cw = np.ascontiguousarray(tri[[0, 2, 1]])
    e1, d1, _ = P.Mesh(cu(xy), cu(tri_cw)).locate_interp(cu(pts))
    e0, d0, _ = mesh.locate_interp(cu(pts))
    e0, d0, e1, d1 = host(e0), host(d0), host(e1), host(d1)
    assert np.array_equal(e0, e1) and np.array_equal(d0, d1)


def test_degenerate_triangles_never_contain(P):
    xy = np.array([[0.0, 1.0, 0.0, 0.5, 2.0], [0.0, 0.0, 1.0, 0.5, 2.0]])
    tri = np.array([[0, 0, 3], [1, 3, 4], [4, 3, 4]], dtype=np.int32)   # #1, #2 collinear/repeated
    pts = np.array([[0.25, 0.5, 0.75, 1.5], [0.25, 0.5, 0.75, 1.5]])
    _check(P, xy, tri, pts, np.arange(5.0))


def test_empty_queries_and_bad_ids(P):
    xy, tri = W.jittered_grid_mesh(4, 0.0)
    mesh = P.Mesh(cu(xy), cu(tri))
    e, d, v = mesh.locate_interp(cu(np.zeros((2, 0))), cu(np.ones(xy.shape[1])))
    assert e.numel() == 0
    bad = tri.copy()
    bad[1, 3] = 999
    with pytest.raises(P.PcmsError) as ex:
        P.Mesh(cu(xy), cu(bad))
    assert ex.value.status == P.INVALID_ARG


def test_full_mesh_config(P):
    """512 x 512 jittered grid (524,288 triangles), 1,000,000 uniform points, f = x^2+3xy."""
    c = W.mesh_2d()
    _check(P, c.xy, c.tri, c.pts, c.field, mode="grid")


@pytest.mark.parametrize("scale", [1.0, 1e-5, 3e4])
def test_points_a_hair_off_the_edges(P, scale):
    """Points displaced from edge midpoints by 1e-16 .. 1e-6 of the edge length, on both sides
    (and exactly on, up to rounding): the orientation signs there are far below what FP32
    resolves, so location must defer to the FP64 filter and the exact expansion and still
    give the oracle's element ids. Meshes at several coordinate scales exercise the FP32
    filter's error allowance, which is proportional to the extent."""
    xy, tri = W.jittered_grid_mesh(48, 0.3, seed=31)
    xy = xy * scale + np.array([[0.25 * scale], [-0.5 * scale]])
    rng = np.random.default_rng(32)
    k = rng.integers(0, tri.shape[1], 3000)
    e = rng.integers(0, 3, 3000)
    a = xy[:, tri[e, k]]
    b = xy[:, tri[(e + 1) % 3, k]]
    t = rng.uniform(0.05, 0.95, 3000)
    base = a + t * (b - a)
    nrm = np.stack([-(b - a)[1], (b - a)[0]])
    eps = 10.0 ** rng.uniform(-16, -6, 3000) * rng.choice([-1.0, 0.0, 1.0], 3000)
    pts = np.concatenate([base + eps * nrm, W.uniform_points(3000, 2, 33) * scale * 0.9], axis=1)
    f = xy[0] / scale + 2 * xy[1] / scale
    _check(P, xy, tri, pts, f, mode="grid")
