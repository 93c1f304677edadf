"""Oracle of the vertex <-> centroid round-trip study (Sec. 3.2.1, Eq. 2 and Eq. 3).

TEST INFRASTRUCTURE ONLY (see the package docstring): called by the tests and by the
benchmark's CPU-baseline leg, never by the product path.

What it computes, each step by its plain definition:
  * element centroids ((v0 + v1) + v2) / 3 of a triangle mesh;
  * the integral of the piecewise-linear (P1) interpolant of nodal values: the sum over
    triangles of |area| times the mean of the three nodal values (exact for P1 functions);
  * the MLS operators vertices -> centroids and centroids -> vertices as the oracle's shape
    functions (QR per target, ``oracle.mls(..., shape=True)``), applied with a sparse
    matrix-vector product;
  * per iteration (one iteration = vertices -> centroids -> vertices), the accuracy error of
    Eq. 2, ||f - f*|| / ||f*|| over the vertices (L2; L-infinity reported too), and the
    conservation error of Eq. 3, |I(f) - I(f*)| / |I(f*)| with I the P1 integral.
Where the paper leaves the norm of Eq. 2 open, L2 over the vertices is the reading used.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def centroids(xy, tri) -> np.ndarray:
    """float64 [2, n_tri]: ((v0 + v1) + v2) / 3 per coordinate."""
    xy = np.asarray(xy, np.float64)
    tri = np.asarray(tri)
    return np.stack([((xy[d][tri[0]] + xy[d][tri[1]]) + xy[d][tri[2]]) / 3.0 for d in range(2)])


def triangle_areas(xy, tri) -> np.ndarray:
    """|((x1-x0)(y2-y0) - (y1-y0)(x2-x0))| / 2 per triangle."""
    x, y = np.asarray(xy[0], np.float64), np.asarray(xy[1], np.float64)
    a, b, c = tri
    cr = (x[b] - x[a]) * (y[c] - y[a]) - (y[b] - y[a]) * (x[c] - x[a])
    return np.abs(cr) * 0.5


def p1_integral(xy, tri, f) -> float:
    """Integral over the mesh of the P1 interpolant of nodal values f."""
    f = np.asarray(f, np.float64)
    a, b, c = tri
    return float(np.sum(triangle_areas(xy, tri) * (((f[a] + f[b]) + f[c]) / 3.0)))


def operator(src, tgt, degree, radius, weight="c4", min_neighbors=0, mode="grid"):
    """The MLS transfer src -> tgt as a sparse matrix (rows: targets), from the oracle's
    shape functions, and the per-target statuses."""
    from oracle import mls
    src = np.ascontiguousarray(src, np.float64)
    o = mls(src, tgt, np.zeros(src.shape[1]), degree, radius, weight=weight,
            min_neighbors=min_neighbors, mode=mode, shape=True)
    off = o["offsets"]
    nt, ns = np.shape(tgt)[1], src.shape[1]
    A = sp.csr_matrix((o["shape"], o["cols"], off), shape=(nt, ns))
    return A, o["status"]


def round_trip(xy, tri, f_star, degree, radius, weight="c4", iterations=1, min_neighbors=0,
               mode="grid") -> dict:
    """Iterate vertices -> centroids -> vertices. Returns dict(accuracy_l2, accuracy_linf,
    conservation: float64[iterations], fields: float64[iterations, n_vertices],
    integral_star, status_v2c, status_c2v)."""
    xy = np.ascontiguousarray(xy, np.float64)
    f_star = np.asarray(f_star, np.float64)
    cen = centroids(xy, tri)
    A, st_a = operator(xy, cen, degree, radius, weight, min_neighbors, mode)
    B, st_b = operator(cen, xy, degree, radius, weight, min_neighbors, mode)
    i_star = p1_integral(xy, tri, f_star)
    n_star2 = np.linalg.norm(f_star)
    n_starinf = np.abs(f_star).max()
    acc2 = np.empty(iterations)
    accinf = np.empty(iterations)
    cons = np.empty(iterations)
    fields = np.empty((iterations, f_star.shape[0]))
    f = f_star.copy()
    for k in range(iterations):
        f = B @ (A @ f)
        fields[k] = f
        acc2[k] = np.linalg.norm(f - f_star) / n_star2
        accinf[k] = np.abs(f - f_star).max() / n_starinf
        cons[k] = abs(p1_integral(xy, tri, f) - i_star) / abs(i_star)
    return dict(accuracy_l2=acc2, accuracy_linf=accinf, conservation=cons, fields=fields,
                integral_star=i_star, status_v2c=st_a, status_c2v=st_b)
