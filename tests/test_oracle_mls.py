"""Pins for the oracle's MLS part (Sec. 3.2.1, Eq. 1, Table 1).

Each test ties the oracle to something other than itself: closed-form values, exact
dyadic geometry, numpy's least-squares / linear solvers on the same systems, the
reproduction and moment properties the method guarantees, and brute force on tiny
inputs. No GPU is used.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2510_18838_gb300 import workloads as W
from tests._helpers import table1_cases

pytestmark = pytest.mark.filterwarnings("ignore")


# ---------------------------------------------------------------- weights (Table 1)
@pytest.mark.parametrize("kind,q,expect", table1_cases())
def test_weight_table_values(orc, kind, q, expect):
    assert orc.weight(kind, q) == pytest.approx(expect, rel=1e-15, abs=1e-300)


# ---------------------------------------------------------------- selection
def _numpy_neighbors(src, tgt, r):
    out = []
    for i in range(tgt.shape[1]):
        d2 = np.zeros(src.shape[1])
        for d in range(src.shape[0]):
            dd = src[d] - tgt[d, i]
            d2 = d2 + dd * dd
        out.append(np.nonzero(d2 < r * r)[0])
    return out


@pytest.mark.parametrize("dim", [2, 3, 4, 5])
def test_neighbors_brute_force_tiny(orc, dim):
    src = W.uniform_points(300, dim, 7)
    tgt = W.uniform_points(40, dim, 8)
    r = {2: 0.2, 3: 0.2, 4: 0.35, 5: 0.45}[dim]
    off, cols, kexp = orc.neighbors(src, tgt, r)
    ref = _numpy_neighbors(src, tgt, r)
    assert (kexp == 0).all()
    for i in range(tgt.shape[1]):
        assert np.array_equal(cols[off[i]:off[i + 1]], ref[i])


def test_neighbors_exact_boundary_dyadic(orc):
    # distances exactly equal to r are excluded (Table 1: phi = 0 for r >= r_c reading)
    t = np.array([[0.5], [0.5]])
    eps = 2.0 ** -40
    src = np.array([[0.75, 0.75 - eps, 0.5, 0.5, 0.25, 0.5 + 0.375, 0.5 + 0.375 - eps],
                    [0.5, 0.5, 0.75, 0.25 + eps, 0.5, 0.5 + 0.5, 0.5 + 0.5]])
    # r = 0.25 for the first five; 3-4-5 triangle (0.375, 0.5) has length 0.625 exactly
    off, cols, _ = orc.neighbors(src, t, 0.25)
    assert cols.tolist() == [1, 3]
    off, cols, _ = orc.neighbors(src, t, 0.625)
    assert 5 not in cols.tolist() and 6 in cols.tolist()


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_mode_matches_brute(orc, dim):
    src = W.uniform_points(3000, dim, 11)
    tgt = W.uniform_points(500, dim, 12, lo=-0.1, hi=1.1)   # some targets outside
    r = 0.07 if dim == 2 else 0.12
    a = orc.neighbors(src, tgt, r, min_neighbors=12, degree=2)
    b = orc.neighbors(src, tgt, r, min_neighbors=12, degree=2, mode="grid")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_min_neighbor_growth_is_minimal_doubling(orc):
    src = W.uniform_points(400, 2, 21)
    tgt = W.uniform_points(60, 2, 22, lo=-0.3, hi=1.3)
    r = 0.02
    off, cols, kexp = orc.neighbors(src, tgt, r, min_neighbors=9, degree=1)
    for i in range(tgt.shape[1]):
        counts = [len(_numpy_neighbors(src, tgt[:, i:i + 1], r * 2.0 ** k)[0]) for k in range(12)]
        k_ref = next(k for k, c in enumerate(counts) if c >= 9)
        assert kexp[i] == k_ref
        assert off[i + 1] - off[i] == counts[k_ref]


@pytest.mark.parametrize("mode", ["brute", "grid"])
def test_global_growth_is_the_smallest_shared_doubling(orc, mode):
    """Global reading of the growth rule: brute-force counts (numpy) at r 2^k for every
    target; K is the first k at which no target is short, and it equals the largest
    per-target doubling (counts only grow with the radius)."""
    src = W.uniform_points(400, 2, 31)
    tgt = W.uniform_points(50, 2, 32, lo=-0.4, hi=1.4)
    r, need = 0.015, 9
    K = orc.global_doublings(src, tgt, r, min_neighbors=need, degree=1, mode=mode)
    counts = np.array([[len(_numpy_neighbors(src, tgt[:, i:i + 1], r * 2.0 ** k)[0])
                        for i in range(tgt.shape[1])] for k in range(K + 1)])
    assert (counts[K] >= need).all()
    assert K > 0 and (counts[K - 1] < need).any()
    _, _, kexp = orc.neighbors(src, tgt, r, min_neighbors=need, degree=1, mode=mode)
    assert K == kexp.max()
    off, cols, kg = orc.neighbors(src, tgt, r, min_neighbors=need, degree=1, mode=mode,
                                  growth="global")
    assert (kg == K).all()
    for i in range(tgt.shape[1]):
        ref = _numpy_neighbors(src, tgt[:, i:i + 1], r * 2.0 ** K)[0]
        assert np.array_equal(cols[off[i]:off[i + 1]], ref)


def test_global_growth_fit_uses_the_shared_radius(orc):
    """A global-growth fit of a quadratic field with a linear basis equals the per-target
    fit at the shared radius (the basis scale and the weights follow that radius), and
    differs from the per-target growth fit where a target needed fewer doublings."""
    src = W.uniform_points(300, 2, 41)
    tgt = W.uniform_points(40, 2, 42, lo=-0.3, hi=1.3)
    f = (src[0] ** 2 + src[0] * src[1])[None]
    r, need = 0.02, 8
    K = orc.global_doublings(src, tgt, r, min_neighbors=need, degree=1)
    g = orc.mls(src, tgt, f, 1, r, min_neighbors=need, growth="global")
    fixed = orc.mls(src, tgt, f, 1, r * 2.0 ** K)
    assert (g["kexp"] == K).all()
    assert np.array_equal(g["values"], fixed["values"])
    per = orc.mls(src, tgt, f, 1, r, min_neighbors=need)
    lower = per["kexp"] < K
    assert lower.any()
    assert not np.allclose(g["values"][0, lower], per["values"][0, lower])


def test_growth_mode_is_checked(orc):
    src = W.uniform_points(20, 2, 1)
    with pytest.raises(ValueError):
        orc.neighbors(src, src, 0.1, min_neighbors=3, growth="sometimes")


# ---------------------------------------------------------------- the fit (Eq. 1)
def _monomials(dim, degree):
    return [e for e in itertools.product(range(degree + 1), repeat=dim) if sum(e) <= degree]


def _poly(pts, expo, centre):
    v = np.ones(pts.shape[1])
    for d, e in enumerate(expo):
        v = v * (pts[d] - centre[d]) ** e
    return v


@pytest.mark.parametrize("dim,degree", [(2, 0), (2, 1), (2, 2), (3, 1), (3, 2), (4, 1), (4, 2),
                                        (5, 1), (5, 2)])
def test_polynomial_reproduction(orc, dim, degree):
    """Every polynomial of degree <= k is reproduced exactly (lambda = 0)."""
    src = W.uniform_points({2: 2500, 3: 6000, 4: 6000, 5: 6000}[dim], dim, 31)
    tgt = W.uniform_points(200 if dim <= 3 else 60, dim, 32, lo=0.1, hi=0.9)
    r = {2: 0.12, 3: 0.25, 4: 0.4, 5: 0.5}[dim]
    centre = [0.3, 0.6, 0.45, 0.55, 0.4][:dim]
    fields = np.stack([_poly(src, e, centre) for e in _monomials(dim, degree)])
    o = orc.mls(src, tgt, fields, degree, r)
    assert (o["status"] == 0).all()
    exact = np.stack([_poly(tgt, e, centre) for e in _monomials(dim, degree)])
    np.testing.assert_allclose(o["values"], exact, rtol=0, atol=1e-12)


def test_linear_basis_does_not_reproduce_quadratics(orc):
    src = W.uniform_points(2500, 2, 33)
    tgt = W.uniform_points(100, 2, 34, lo=0.1, hi=0.9)
    f = (src[0] - 0.5) ** 2
    o = orc.mls(src, tgt, f, 1, 0.12)
    assert np.abs(o["values"][0] - (tgt[0] - 0.5) ** 2).max() > 1e-4


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 2), (5, 2)])
def test_partition_of_unity_and_moments(orc, dim, degree):
    """Shape functions satisfy sum_j N_j p(s_j - t) = e_1 for the whole basis."""
    src = W.uniform_points({2: 2000, 3: 5000, 5: 5000}[dim], dim, 41)
    tgt = W.uniform_points(80 if dim <= 3 else 30, dim, 42)
    r = {2: 0.12, 3: 0.25, 5: 0.5}[dim]
    o = orc.mls(src, tgt, np.zeros((1, src.shape[1])), degree, r, shape=True, min_neighbors=15)
    off, cols, shp = o["offsets"], o["cols"], o["shape"]
    for i in range(tgt.shape[1]):
        nb = cols[off[i]:off[i + 1]]
        N = shp[off[i]:off[i + 1]]
        for e in _monomials(dim, degree):
            mom = np.sum(N * _poly(src[:, nb], e, tgt[:, i]))
            assert mom == pytest.approx(1.0 if sum(e) == 0 else 0.0, abs=1e-12)


def test_shape_functions_reproduce_values(orc):
    c = W.mls_2d_small(3000, 300)
    o = orc.mls(c.src, c.tgt, c.fields, 2, 0.06, shape=True)
    off, cols, shp = o["offsets"], o["cols"], o["shape"]
    ok = o["status"] == 0
    assert ok.sum() > 250
    v = np.array([np.sum(shp[off[i]:off[i + 1]] * c.fields[0, cols[off[i]:off[i + 1]]])
                  for i in range(c.tgt.shape[1])])
    np.testing.assert_allclose(v[ok], o["values"][0][ok], rtol=0, atol=1e-13)


def test_degree0_is_shepard(orc):
    src = W.uniform_points(1500, 2, 51)
    tgt = W.uniform_points(100, 2, 52)
    f = np.cos(3 * src[0]) + src[1]
    r = 0.1
    o = orc.mls(src, tgt, f, 0, r)
    nb = _numpy_neighbors(src, tgt, r)
    for i in range(tgt.shape[1]):
        d = np.sqrt(((src[:, nb[i]] - tgt[:, i:i + 1]) ** 2).sum(0)) / r
        w = np.array([orc.weight("wendland_c2", q) for q in d])
        if len(nb[i]) == 0:
            assert o["status"][i] == 1
            continue
        assert o["values"][0, i] == pytest.approx(np.sum(w * f[nb[i]]) / np.sum(w), rel=1e-13)


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 2), (4, 2), (5, 1), (5, 2)])
def test_const_weight_equals_plain_lstsq_uncentred(orc, dim, degree):
    """Constant weight -> ordinary least squares; evaluated with the raw, uncentred
    monomials (numpy lstsq), which also pins the centring/scaling of the basis."""
    src = W.uniform_points({2: 1500, 3: 4000, 4: 4000, 5: 4000}[dim], dim, 61)
    tgt = W.uniform_points(50 if dim <= 3 else 20, dim, 62, lo=0.2, hi=0.8)
    f = np.exp(src[0]) * np.sin(2 * src[1])
    r = {2: 0.1, 3: 0.2, 4: 0.35, 5: 0.45}[dim]
    o = orc.mls(src, tgt, f, degree, r, weight="const")
    nb = _numpy_neighbors(src, tgt, r)
    mons = _monomials(dim, degree)
    for i in range(tgt.shape[1]):
        A = np.stack([_poly(src[:, nb[i]], e, [0.0] * dim) for e in mons], axis=1)
        c, *_ = np.linalg.lstsq(A, f[nb[i]], rcond=None)
        val = sum(ck * _poly(tgt[:, i:i + 1], e, [0.0] * dim)[0] for ck, e in zip(c, mons))
        assert o["values"][0, i] == pytest.approx(val, rel=1e-9, abs=1e-11)


def test_weighted_lstsq_matches_numpy(orc):
    src = W.uniform_points(2000, 2, 71)
    tgt = W.uniform_points(60, 2, 72)
    f = np.sin(5 * src[0]) * src[1]
    r = 0.1
    for kind in ["wendland_c2", "gaussian", "c4", "imq", "mq"]:
        o = orc.mls(src, tgt, f, 2, r, weight=kind)
        nb = _numpy_neighbors(src, tgt, r)
        for i in range(tgt.shape[1]):
            if len(nb[i]) < 6:
                continue
            u = (src[:, nb[i]] - tgt[:, i:i + 1]) / r
            q = np.sqrt(((src[:, nb[i]] - tgt[:, i:i + 1]) ** 2).sum(0)) / r
            w = np.array([orc.weight(kind, x) for x in q])
            A = np.stack([np.ones_like(u[0]), u[0], u[1], u[0] ** 2, u[0] * u[1], u[1] ** 2], 1)
            sw = np.sqrt(w)
            c, *_ = np.linalg.lstsq(sw[:, None] * A, sw * f[nb[i]], rcond=None)
            assert o["values"][0, i] == pytest.approx(c[0], rel=1e-10, abs=1e-12), kind


def test_tikhonov_matches_augmented_lstsq(orc):
    src = W.uniform_points(1500, 2, 81)
    tgt = W.uniform_points(40, 2, 82)
    f = np.cos(4 * src[0] + src[1])
    r, lam = 0.1, 0.3
    o = orc.mls(src, tgt, f, 2, r, lam=lam)
    nb = _numpy_neighbors(src, tgt, r)
    for i in range(tgt.shape[1]):
        if len(nb[i]) < 6:
            continue
        u = (src[:, nb[i]] - tgt[:, i:i + 1]) / r
        q = np.sqrt((u ** 2).sum(0))
        w = np.array([orc.weight("wendland_c2", x) for x in q])
        A = np.stack([np.ones_like(u[0]), u[0], u[1], u[0] ** 2, u[0] * u[1], u[1] ** 2], 1)
        sw = np.sqrt(w)
        Aa = np.vstack([sw[:, None] * A, math.sqrt(lam) * np.eye(6)])
        ba = np.concatenate([sw * f[nb[i]], np.zeros(6)])
        c, *_ = np.linalg.lstsq(Aa, ba, rcond=None)
        assert o["values"][0, i] == pytest.approx(c[0], rel=1e-10, abs=1e-12)


def test_exactly_m_points_is_interpolation(orc):
    """|N| = m with non-degenerate points: the fit interpolates, independent of weights."""
    rng = np.random.default_rng(91)
    for trial in range(20):
        t = np.array([[0.5], [0.5]])
        ang = np.sort(rng.uniform(0, 2 * np.pi, 6))
        rad = rng.uniform(0.2, 0.9, 6) * 0.1
        src = np.stack([0.5 + rad * np.cos(ang), 0.5 + rad * np.sin(ang)])
        f = rng.standard_normal(6)
        o1 = orc.mls(src, t, f, 2, 0.1)
        o2 = orc.mls(src, t, f, 2, 0.1, weight="gaussian")
        A = np.stack([np.ones(6), src[0], src[1], src[0] ** 2, src[0] * src[1], src[1] ** 2], 1)
        c = np.linalg.solve(A, f)
        val = c @ np.array([1, 0.5, 0.5, 0.25, 0.25, 0.25])
        assert o1["values"][0, 0] == pytest.approx(val, rel=1e-8, abs=1e-9)
        assert o2["values"][0, 0] == pytest.approx(val, rel=1e-8, abs=1e-9)


def test_translation_and_axis_permutation_invariance(orc):
    src = W.uniform_points(2000, 3, 95)
    tgt = W.uniform_points(60, 3, 96)
    f = np.sin(3 * src[0]) + src[1] * src[2]
    base = orc.mls(src, tgt, f, 2, 0.25)["values"]
    shift = np.array([[0.25], [-0.5], [1.0]])    # dyadic: coordinate differences stay exact
    moved = orc.mls(src + shift, tgt + shift, f, 2, 0.25)["values"]
    np.testing.assert_allclose(moved, base, rtol=0, atol=1e-12)
    perm = [2, 0, 1]
    swapped = orc.mls(src[perm], tgt[perm], f, 2, 0.25)["values"]
    np.testing.assert_allclose(swapped, base, rtol=0, atol=1e-12)


def test_underdetermined_status_and_nan(orc):
    src = np.array([[0.5, 0.52, 0.9], [0.5, 0.5, 0.9]])
    tgt = np.array([[0.5, 0.9, 0.1], [0.5, 0.9, 0.1]])
    o = orc.mls(src, tgt, np.ones(3), 1, 0.05)
    assert o["status"].tolist() == [1, 1, 1]
    assert np.isnan(o["values"]).all()
    o = orc.mls(src, tgt, np.ones(3), 0, 0.05)      # Shepard needs one point
    assert o["status"].tolist() == [0, 0, 1]
    np.testing.assert_allclose(o["values"][0, :2], [1.0, 1.0], rtol=0, atol=1e-15)


def test_collinear_points_are_ill_conditioned(orc):
    x = np.linspace(0.4, 0.6, 15)
    src = np.stack([x, 0.5 + 0.25 * (x - 0.5)])            # all on one line
    tgt = np.array([[0.5], [0.5]])
    for deg in (1, 2):
        o = orc.mls(src, tgt, np.ones(15), deg, 0.2)
        assert o["status"][0] == 2 and np.isnan(o["values"][0, 0])
    o = orc.mls(src, tgt, 1.0 + x, 0, 0.2)                  # Shepard is fine
    assert o["status"][0] == 0
    # a quadratic basis on points of a circle is singular too (x^2 + y^2 = const)
    ang = np.linspace(0, 2 * np.pi, 20, endpoint=False)
    src = np.stack([0.5 + 0.05 * np.cos(ang), 0.5 + 0.05 * np.sin(ang)])
    o = orc.mls(src, tgt, np.ones(20), 2, 0.2)
    assert o["status"][0] == 2
    o = orc.mls(src, tgt, np.ones(20), 1, 0.2)
    assert o["status"][0] == 0


def test_selection_excludes_nonpositive_weights(orc):
    """Selection is phi > 0 (Sec. 3.2.1): TPS with a = 2 is <= 0 for r <= r_c / 2."""
    src = np.array([[0.5, 0.5 + 0.1, 0.5 + 0.3, 0.5 + 0.45], [0.5] * 4])
    t = np.array([[0.5], [0.5]])
    _, cols, _ = orc.neighbors(src, t, 0.5, weight="tps")
    assert cols.tolist() == [2, 3]
    _, cols, _ = orc.neighbors(src, t, 0.5, weight="cubic")
    assert cols.tolist() == [1, 2, 3]
    _, cols, _ = orc.neighbors(src, t, 0.5, weight="wendland_c2")
    assert cols.tolist() == [0, 1, 2, 3]
