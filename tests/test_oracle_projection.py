"""Pins for the oracle of the conservative L2 projection (Sec. 3.2.2, mesh intersection).

Closed forms for the clipping and the mass matrix, and the properties the projection has by
construction: the P1 space of the target reproduces linear source fields exactly, the integral
is conserved, the supermesh tiles the common domain, and projecting onto the same mesh is the
identity.
"""
import numpy as np
import pytest

import oracle
from oracle import projection as PR
from paper_2510_18838_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


def _area(poly):
    x = np.array([p[0] for p in poly])
    y = np.array([p[1] for p in poly])
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_clip_closed_forms():
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    # a copy shifted by (1/2, 0): the overlap is the triangle (1/2,0), (1,0), (1/2,1/2)
    shifted = tri + np.array([0.5, 0.0])
    assert _area(PR.clip_triangle(shifted, tri)) == pytest.approx(0.125, abs=1e-15)
    # the other half of the unit square: the two triangles share only the diagonal
    refl = np.array([[1.0, 1.0], [0.0, 1.0], [1.0, 0.0]])
    assert _area(PR.clip_triangle(refl, tri)) == pytest.approx(0.0, abs=1e-15)
    # a small triangle inside is returned whole; a far one gives nothing
    small = np.array([[0.1, 0.1], [0.3, 0.1], [0.1, 0.3]])
    assert _area(PR.clip_triangle(small, tri)) == pytest.approx(0.02, abs=1e-15)
    assert PR.clip_triangle(small + 5.0, tri) == []
    # two opposite equilateral triangles inscribed in the unit circle (a hexagram): their
    # intersection is the regular hexagon of side r / sqrt(3)
    r = 1.0
    up = np.array([[r * np.cos(a), r * np.sin(a)] for a in np.pi / 2 + np.arange(3) * 2 * np.pi / 3])
    dn = -up
    hexa = PR.clip_triangle(dn, up)
    assert len(hexa) == 6
    assert _area(hexa) == pytest.approx(3 * np.sqrt(3) / 2 * (r / np.sqrt(3)) ** 2, rel=1e-13)


def test_mass_matrix_closed_form():
    xy = np.array([[0.0, 2.0, 0.0], [0.0, 0.0, 3.0]])    # one triangle of area 3
    tri = np.array([[0], [1], [2]])
    M = PR.mass_matrix(xy, tri).toarray()
    np.testing.assert_allclose(M, 3.0 / 12.0 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]),
                               rtol=0, atol=1e-15)
    xs, ts = W.jittered_grid_mesh(9, 0.3, 2)
    M = PR.mass_matrix(xs, ts)
    assert M.sum() == pytest.approx(1.0, abs=1e-14)          # sum N_A N_B = 1 over the square
    np.testing.assert_allclose(M.toarray(), M.toarray().T, rtol=0, atol=0)


@pytest.mark.parametrize("ns,nt", [(11, 17), (16, 7)])
def test_projection_reproduces_linear_fields_and_conserves(ns, nt):
    xs, ts = W.jittered_grid_mesh(ns, 0.3, 3)
    xt, tt = W.jittered_grid_mesh(nt, 0.3, 4)
    f = 1.0 + 2.0 * xs[0] - 3.0 * xs[1]
    o = oracle.l2_projection(xs, ts, f, xt, tt)
    np.testing.assert_allclose(o["values"], 1.0 + 2.0 * xt[0] - 3.0 * xt[1], rtol=0, atol=1e-13)
    assert o["supermesh_area"] == pytest.approx(1.0, abs=1e-13)
    g = np.sin(3 * xs[0]) * np.cos(2 * xs[1]) + 2.0
    o = oracle.l2_projection(xs, ts, g, xt, tt)
    assert abs(o["integral_target"] - o["integral_source"]) <= 1e-13
    # the right-hand side of f = 1 is the row sums of the target's mass matrix (sum_B N_B = 1)
    one = oracle.l2_projection(xs, ts, np.ones(xs.shape[1]), xt, tt)
    np.testing.assert_allclose(one["rhs"], np.asarray(PR.mass_matrix(xt, tt).sum(1)).ravel(),
                               rtol=0, atol=1e-14)


def test_projection_onto_the_same_mesh_is_the_identity():
    xs, ts = W.jittered_grid_mesh(12, 0.3, 6)
    g = np.exp(xs[0]) * np.sin(4 * xs[1])
    o = oracle.l2_projection(xs, ts, g, xs, ts)
    np.testing.assert_allclose(o["values"], g, rtol=0, atol=1e-13)


def test_projection_of_a_quadratic_is_not_exact_but_close():
    xs, ts = W.jittered_grid_mesh(20, 0.3, 3)
    xt, tt = W.jittered_grid_mesh(13, 0.3, 4)
    f = xs[0] ** 2 + xs[1] ** 2
    o = oracle.l2_projection(xs, ts, f, xt, tt)
    err = np.abs(o["values"] - (xt[0] ** 2 + xt[1] ** 2)).max()
    assert 1e-5 < err < 1e-2
