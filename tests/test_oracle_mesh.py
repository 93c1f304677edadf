"""Pins for the oracle's mesh part (Sec. 3.3: point localization, lowest-order
classification, parametric/barycentric interpolation).

Orientation signs are checked against exact rational arithmetic; element ids on an
unjittered grid against their closed form, including points on edges and vertices
(dyadic coordinates, so every test point is exact); interpolation against linear fields.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2510_18838_gb300 import workloads as W


def _sign_fraction(a, b, c):
    ax, ay = map(Fraction, a)
    bx, by = map(Fraction, b)
    cx, cy = map(Fraction, c)
    d = (ax - cx) * (by - cy) - (ay - cy) * (bx - cx)
    return (d > 0) - (d < 0)


def test_orient2d_exact_random_and_degenerate(orc):
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(3000):
        cases.append(tuple(map(tuple, rng.uniform(-1, 1, (3, 2)))))
    # nearly collinear: c = a + t (b - a) rounded, then nudged by a few ulps
    for _ in range(3000):
        a = rng.uniform(-1, 1, 2)
        b = rng.uniform(-1, 1, 2)
        t = rng.uniform(-2, 3)
        c = a + t * (b - a)
        k = rng.integers(-3, 4)
        c = c.copy()
        c[0] = np.nextafter(c[0], np.inf) if k > 0 else (np.nextafter(c[0], -np.inf) if k < 0 else c[0])
        cases.append((tuple(a), tuple(b), tuple(c)))
    # exactly collinear dyadic points and repeated points
    cases += [((0.0, 0.0), (1.0, 1.0), (0.5, 0.5)), ((0.125, 0.25), (0.125, 0.25), (3.0, 1.0)),
              ((12.0, 12.0), (24.0, 24.0), (0.5, 0.5)), ((0.5, 0.5), (12.0, 12.0), (24.0, 24.0))]
    # the classic hard case: (0.5 + i 2^-53, 0.5 + j 2^-53) against (12,12)-(24,24)
    for i in range(16):
        for j in range(16):
            p = (0.5 + i * 2.0 ** -53, 0.5 + j * 2.0 ** -53)
            cases.append((p, (12.0, 12.0), (24.0, 24.0)))
    got = [orc.orient2d_sign(*c) for c in cases]
    ref = [_sign_fraction(*c) for c in cases]
    assert got == ref
    assert 0 in ref and 1 in ref and -1 in ref


def _closed_form_elem(p, n):
    """Element id on the unjittered n x n grid (diagonal (i,j)-(i+1,j+1)), smallest id
    among all closed triangles containing p; p must be dyadic with denominator n*2^k."""
    px, py = Fraction(p[0]), Fraction(p[1])
    best = None
    for j in range(n):
        for i in range(n):
            lx, ly = px * n - i, py * n - j         # local coords in cell
            if not (0 <= lx <= 1 and 0 <= ly <= 1):
                continue
            cands = []
            if ly <= lx:                              # lower-right: (0,0),(1,0),(1,1)
                cands.append(2 * (j * n + i))
            if ly >= lx:                              # upper-left: (0,0),(1,1),(0,1)
                cands.append(2 * (j * n + i) + 1)
            for c in cands:
                best = c if best is None else min(best, c)
    return -1 if best is None else best


def _closed_form_dim(p, n):
    px, py = Fraction(p[0]) * n, Fraction(p[1]) * n
    on_vx = px.denominator == 1
    on_hy = py.denominator == 1
    on_diag = (px - py).denominator == 1
    k = on_vx + on_hy + on_diag
    return 0 if k >= 2 else (1 if k == 1 else 2)


def test_locate_unjittered_closed_form(orc):
    n = 8
    xy, tri = W.jittered_grid_mesh(n, jitter=0.0)
    rng = np.random.default_rng(3)
    # random dyadic points with denominator 64*n: interior, edges, vertices, diagonals
    pts = rng.integers(0, 64 * n + 1, size=(2, 600)) / (64.0 * n)
    coarse = rng.integers(0, n + 1, size=(2, 100)) / float(n)           # grid vertices
    half = rng.integers(0, 2 * n + 1, size=(2, 100)) / (2.0 * n)       # edge midpoints etc
    pts = np.concatenate([pts, coarse, half, np.array([[-0.25, 1.5], [0.5, 0.5]])], axis=1)
    elem, dimc, _ = orc.locate(xy, tri, pts)
    for k in range(pts.shape[1]):
        p = (pts[0, k], pts[1, k])
        ref = _closed_form_elem(p, n)
        assert elem[k] == ref, (p, elem[k], ref)
        if ref >= 0:
            assert dimc[k] == _closed_form_dim(p, n), p
        else:
            assert dimc[k] == -1


def test_locate_grid_mode_matches_exhaustive(orc):
    xy, tri = W.jittered_grid_mesh(24, 0.3, seed=9)
    pts = W.uniform_points(4000, 2, 10, lo=-0.05, hi=1.05)
    # add vertices and edge midpoints of the jittered mesh (degenerate classifications)
    mid = 0.5 * (xy[:, tri[0, :200]] + xy[:, tri[1, :200]])
    pts = np.concatenate([pts, xy[:, :300], mid], axis=1)
    a = orc.locate(xy, tri, pts)
    b = orc.locate(xy, tri, pts, mode="grid")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert (a[1][4000:4300] == 0).all()            # every vertex classifies on a vertex


def test_generated_mesh_is_ccw_and_conforming(orc):
    xy, tri = W.jittered_grid_mesh(32, 0.3, seed=201)
    s = orc.orient2d_sign(xy[:, tri[0]], xy[:, tri[1]], xy[:, tri[2]])
    assert (s == 1).all()
    # conforming: a strictly interior sample point of each triangle locates to it
    cen = (xy[:, tri[0]] + xy[:, tri[1]] + xy[:, tri[2]]) / 3.0
    elem, dimc, _ = orc.locate(xy, tri, cen, mode="grid")
    assert np.array_equal(elem, np.arange(tri.shape[1])) and (dimc == 2).all()


def test_interpolation_reproduces_linear_fields(orc):
    xy, tri = W.jittered_grid_mesh(20, 0.3, seed=4)
    pts = W.uniform_points(3000, 2, 5)
    for a, b, c in [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (2.5, -3.0, 7.0)]:
        f = a + b * xy[0] + c * xy[1]
        elem, _, v = orc.locate(xy, tri, pts, field=f, mode="grid")
        assert (elem >= 0).all()
        np.testing.assert_allclose(v, a + b * pts[0] + c * pts[1], rtol=0, atol=1e-13)


def test_interpolation_at_vertices_and_outside(orc):
    xy, tri = W.jittered_grid_mesh(10, 0.3, seed=6)
    f = xy[0] ** 2 + 3 * xy[0] * xy[1]
    elem, dimc, v = orc.locate(xy, tri, xy, field=f)
    assert (dimc == 0).all()
    np.testing.assert_allclose(v, f, rtol=0, atol=1e-14)
    out = np.array([[-0.1, 1.2, 0.5], [0.5, 0.5, 1.0000001]])
    elem, dimc, v = orc.locate(xy, tri, out, field=f)
    assert elem.tolist() == [-1, -1, -1] and np.isnan(v).all()


def test_quadratic_field_is_not_reproduced(orc):
    xy, tri = W.jittered_grid_mesh(16, 0.3, seed=8)
    pts = W.uniform_points(500, 2, 9)
    f = xy[0] ** 2 + 3 * xy[0] * xy[1]
    _, _, v = orc.locate(xy, tri, pts, field=f)
    err = np.abs(v - (pts[0] ** 2 + 3 * pts[0] * pts[1])).max()
    assert 1e-6 < err < (1.0 / 16) ** 2 * 4
