"""Oracle of the conservative L2 projection between two 2D triangle meshes (Sec. 3.2.2,
mesh intersection methods).

TEST INFRASTRUCTURE ONLY (see the package docstring).

What it computes, each step by its plain definition, for a P1 (piecewise-linear) source field
f_s on mesh S and P1 shape functions N_A on mesh T:
  * the supermesh: every intersecting pair (source triangle, target triangle) clipped to its
    common convex polygon (Sutherland-Hodgman against the target triangle's three edges),
    found by brute force over all pairs whose bounding boxes overlap;
  * the load vector, entry A the integral of N_A f_s: each polygon split into a fan of triangles,
    each integrated with the three-point edge-midpoint rule (exact for quadratics, so for the
    product of two linear functions);
  * the consistent mass matrix M_AB = integral of N_A N_B (per triangle |T|/12 [2 1 1; 1 2 1;
    1 1 2]) and the projected field f_t = M^-1 b (a sparse direct solve).
Because the N_A sum to one, the integral of f_t equals that of f_s over the covered region:
the projection conserves the integral (Eq. 3's quantity) exactly, up to the solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _orient(ax, ay, bx, by, cx, cy):
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)


def clip_triangle(src, tgt):
    """src, tgt: (3, 2) arrays, tgt counter-clockwise. The polygon src ∩ tgt as a list of
    (x, y), clipped successively by the half-planes left of tgt's edges."""
    poly = [tuple(p) for p in src]
    for k in range(3):
        ax, ay = tgt[k]
        bx, by = tgt[(k + 1) % 3]
        out = []
        n = len(poly)
        for i in range(n):
            px, py = poly[i]
            qx, qy = poly[(i + 1) % n]
            sp_ = _orient(ax, ay, bx, by, px, py)
            sq = _orient(ax, ay, bx, by, qx, qy)
            if sp_ >= 0:
                out.append((px, py))
            if (sp_ >= 0) != (sq >= 0):
                t = sp_ / (sp_ - sq)
                out.append((px + t * (qx - px), py + t * (qy - py)))
        poly = out
        if len(poly) < 3:
            return []
    return poly


def _bary(tri, x, y):
    """Barycentric coordinates of (x, y) in triangle tri (3, 2)."""
    (x0, y0), (x1, y1), (x2, y2) = tri
    det = _orient(x0, y0, x1, y1, x2, y2)
    l1 = _orient(x0, y0, x, y, x2, y2) / det
    l2 = _orient(x0, y0, x1, y1, x, y) / det
    return np.array([1.0 - l1 - l2, l1, l2])


def _ccw(xy, tri):
    t = np.array(tri, dtype=np.int64)
    a, b, c = t
    o = _orient(xy[0][a], xy[1][a], xy[0][b], xy[1][b], xy[0][c], xy[1][c])
    sw = o < 0
    t[1, sw], t[2, sw] = t[2, sw].copy(), t[1, sw].copy()
    return t


def mass_matrix(xy, tri) -> sp.csr_matrix:
    t = _ccw(xy, tri)
    x, y = np.asarray(xy[0]), np.asarray(xy[1])
    area = 0.5 * np.abs(_orient(x[t[0]], y[t[0]], x[t[1]], y[t[1]], x[t[2]], y[t[2]]))
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(t[a])
            cols.append(t[b])
            vals.append(area * (2.0 if a == b else 1.0) / 12.0)
    n = x.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def supermesh_rhs(xs, ts, fs, xt, tt):
    """b_A = integral of N_A f_s over the supermesh, and the supermesh's total area."""
    ts, tt = _ccw(xs, ts), _ccw(xt, tt)
    XS = np.stack([np.asarray(xs[0])[ts], np.asarray(xs[1])[ts]], axis=-1)   # (3, nS, 2)
    XT = np.stack([np.asarray(xt[0])[tt], np.asarray(xt[1])[tt]], axis=-1)
    XS = np.transpose(XS, (1, 0, 2))
    XT = np.transpose(XT, (1, 0, 2))
    smin, smax = XS.min(axis=1), XS.max(axis=1)
    b = np.zeros(np.asarray(xt).shape[1])
    total = 0.0
    for j in range(XT.shape[0]):
        T = XT[j]
        tmin, tmax = T.min(axis=0), T.max(axis=0)
        cand = np.nonzero((smin[:, 0] <= tmax[0]) & (smax[:, 0] >= tmin[0]) &
                          (smin[:, 1] <= tmax[1]) & (smax[:, 1] >= tmin[1]))[0]
        for i in cand:
            S = XS[i]
            poly = clip_triangle(S, T)
            if len(poly) < 3:
                continue
            p0 = poly[0]
            for k in range(1, len(poly) - 1):
                p1, p2 = poly[k], poly[k + 1]
                ar = 0.5 * abs(_orient(p0[0], p0[1], p1[0], p1[1], p2[0], p2[1]))
                if ar == 0.0:
                    continue
                total += ar
                for (ax, ay), (bx, by) in ((p0, p1), (p1, p2), (p2, p0)):
                    mx, my = 0.5 * (ax + bx), 0.5 * (ay + by)
                    ns = _bary(S, mx, my)
                    nt = _bary(T, mx, my)
                    fv = float(ns @ fs[ts[:, i]])
                    b[tt[:, j]] += (ar / 3.0) * nt * fv
    return b, total


def l2_projection(xs, ts, fs, xt, tt) -> dict:
    """Project the P1 field fs (nodal, on mesh (xs, ts)) onto the P1 space of mesh (xt, tt).
    Returns dict(values, rhs, supermesh_area, integral_source, integral_target)."""
    from oracle.roundtrip import p1_integral
    fs = np.asarray(fs, np.float64)
    b, area = supermesh_rhs(xs, ts, fs, xt, tt)
    M = mass_matrix(xt, tt).tocsc()
    f = spla.spsolve(M, b)
    return dict(values=f, rhs=b, supermesh_area=area,
                integral_source=p1_integral(xs, ts, fs), integral_target=p1_integral(xt, tt, f))
