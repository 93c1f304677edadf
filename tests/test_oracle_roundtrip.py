"""Pins for the oracle of the vertex <-> centroid round trip (Sec. 3.2.1, Eq. 2 and Eq. 3).

The P1 integral is pinned by closed forms (it is exact for linear fields), the centroids by
the closed form of the unjittered grid, and the round trip by the reproduction property of
the fit (fields in the basis's span come back unchanged, iteration after iteration).
"""
import numpy as np
import pytest

import oracle
from paper_2510_18838_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


def _west_box(xy):
    """The unit-square mesh stretched to [1.8, 3.2] x [-0.8, 0.8] (a tokamak R-Z box)."""
    return np.stack([1.8 + 1.4 * xy[0], -0.8 + 1.6 * xy[1]])


@pytest.mark.parametrize("box", [False, True])
def test_p1_integral_of_linear_fields_is_exact(box):
    xy, tri = W.jittered_grid_mesh(24, 0.3, 11)
    if box:
        xy = _west_box(xy)
        area, xm, ym = 1.4 * 1.6, 2.5, 0.0
    else:
        area, xm, ym = 1.0, 0.5, 0.5
    for a, b, c in [(1.0, 0.0, 0.0), (0.3, -2.0, 0.7), (-1.5, 0.25, 3.0)]:
        f = a + b * xy[0] + c * xy[1]
        assert oracle.p1_integral(xy, tri, f) == pytest.approx(area * (a + b * xm + c * ym),
                                                               rel=1e-13, abs=1e-13)


def test_p1_integral_of_a_quadratic_on_the_unjittered_grid():
    """On the regular grid the P1 interpolant of x^2 overshoots by h^2/6 on every cell (the
    chord above the parabola on each triangle edge along x): integral 1/3 + h^2/6."""
    n = 16
    xy, tri = W.jittered_grid_mesh(n, 0.0, 1)
    h = 1.0 / n
    assert oracle.p1_integral(xy, tri, xy[0] ** 2) == pytest.approx(1.0 / 3.0 + h * h / 6.0,
                                                                    rel=1e-13)


def test_centroids_closed_form_on_the_unjittered_grid():
    n = 8
    xy, tri = W.jittered_grid_mesh(n, 0.0, 1)
    c = oracle.centroids(xy, tri)
    h = 1.0 / n
    k = np.arange(n * n)
    i, j = k % n, k // n
    np.testing.assert_allclose(c[0, 0::2], (3 * i + 2) * h / 3, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c[1, 0::2], (3 * j + 1) * h / 3, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c[0, 1::2], (3 * i + 1) * h / 3, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c[1, 1::2], (3 * j + 2) * h / 3, rtol=0, atol=1e-15)


@pytest.mark.parametrize("degree", [1, 2])
def test_round_trip_reproduces_fields_in_the_basis(degree):
    n = 20
    xy, tri = W.jittered_grid_mesh(n, 0.3, 5)
    xy = _west_box(xy)
    f = 2.0 + 0.5 * xy[0] - 1.5 * xy[1]
    if degree == 2:
        f = f + 0.3 * xy[0] ** 2 - 0.8 * xy[0] * xy[1] + 0.2 * xy[1] ** 2
    o = oracle.round_trip(xy, tri, f, degree, 2.5 * 1.6 / n, iterations=4)
    assert (o["status_v2c"] == 0).all() and (o["status_c2v"] == 0).all()
    assert o["accuracy_l2"].max() <= 1e-13
    assert o["accuracy_linf"].max() <= 1e-13
    assert o["conservation"].max() <= 1e-13


def test_linear_round_trip_does_not_reproduce_quadratics():
    n = 20
    xy, tri = W.jittered_grid_mesh(n, 0.3, 5)
    f = xy[0] ** 2 + xy[1] ** 2
    o = oracle.round_trip(xy, tri, f, 1, 2.5 / n, iterations=2)
    assert o["accuracy_l2"][0] > 1e-6
    assert o["accuracy_l2"][1] > o["accuracy_l2"][0]


def test_round_trip_errors_of_the_smooth_field():
    """The study's field sin(x)cos(y) + 2: both errors are small and grow with the
    iterations, each iteration adding a similar amount (the behaviour the study reports)."""
    n = 24
    xy, tri = W.jittered_grid_mesh(n, 0.3, 9)
    xy = _west_box(xy)
    f = np.sin(xy[0]) * np.cos(xy[1]) + 2.0
    o = oracle.round_trip(xy, tri, f, 1, 2.5 * 1.6 / n, iterations=6)
    acc = o["accuracy_l2"]
    assert 0 < acc[0] < 1e-2
    assert (np.diff(acc) > 0).all()
    inc = np.diff(np.concatenate([[0.0], acc]))
    assert inc.max() / inc.min() < 2.0
