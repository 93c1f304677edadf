"""GPU parity of the conservative L2 projection between 2D meshes (Sec. 3.2.2) against the
oracle: projected values within the FP64 tolerance, exact reproduction of linear fields,
conservation of the integral, the supermesh area, and the identity on a shared mesh.
Every call goes through the C ABI."""
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


def _mesh(P, xy, tri):
    import torch
    return P.Mesh(torch.from_numpy(np.ascontiguousarray(xy)).cuda(),
                  torch.from_numpy(np.ascontiguousarray(tri)).cuda())


def _cu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


@pytest.mark.parametrize("ns,nt,shift", [(13, 17, 0.0), (24, 9, 0.0), (16, 16, 0.0),
                                         (12, 15, 0.23)])
def test_projection_matches_oracle(P, ns, nt, shift):
    xs, ts = W.jittered_grid_mesh(ns, 0.3, 30 + ns)
    xt, tt = W.jittered_grid_mesh(nt, 0.3, 40 + nt)
    xt = np.ascontiguousarray(xt + shift)          # partly outside the source domain
    g = np.sin(3 * xs[0]) * np.cos(2 * xs[1]) + 2.0
    S, T = _mesh(P, xs, ts), _mesh(P, xt, tt)
    f, info = P.l2_project(S, _cu(g), T)
    o = oracle.l2_projection(xs, ts, g, xt, tt)
    assert normwise_err(f.cpu().numpy()[None], o["values"][None]) <= TOL_FP64
    assert info["supermesh_area"] == pytest.approx(o["supermesh_area"], rel=1e-13, abs=1e-15)
    assert info["relative_residual"] <= 1e-14
    # conservation: the P1 integral of the projection equals the source's over the overlap
    assert abs(T.integrate(f) - o["integral_target"]) <= 1e-13
    if shift == 0.0:
        assert abs(T.integrate(f) - S.integrate(_cu(g))) <= 1e-13
    S.destroy()
    T.destroy()


def test_linear_fields_are_reproduced_and_identity(P):
    xs, ts = W.jittered_grid_mesh(21, 0.3, 5)
    xt, tt = W.jittered_grid_mesh(14, 0.3, 6)
    S, T = _mesh(P, xs, ts), _mesh(P, xt, tt)
    f, info = P.l2_project(S, _cu(1.0 + 2.0 * xs[0] - 3.0 * xs[1]), T)
    np.testing.assert_allclose(f.cpu().numpy(), 1.0 + 2.0 * xt[0] - 3.0 * xt[1], rtol=0,
                               atol=1e-12)
    assert info["supermesh_area"] == pytest.approx(1.0, abs=1e-13)
    g = np.exp(xs[0]) * np.sin(4 * xs[1])
    same, _ = P.l2_project(S, _cu(g), S)
    np.testing.assert_allclose(same.cpu().numpy(), g, rtol=0, atol=1e-12)
    S.destroy()
    T.destroy()


def test_projection_is_reproducible(P):
    xs, ts = W.jittered_grid_mesh(30, 0.3, 7)
    xt, tt = W.jittered_grid_mesh(41, 0.3, 8)
    g = np.cos(5 * xs[0] * xs[1])
    S, T = _mesh(P, xs, ts), _mesh(P, xt, tt)
    a, _ = P.l2_project(S, _cu(g), T)
    b, _ = P.l2_project(S, _cu(g), T)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    S.destroy()
    T.destroy()
