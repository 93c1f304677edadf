"""CPU check of the CUDA library's per-target MLS algebra (moment accumulation, monomial
tables, guarded LDL^T solve, the re-centred basis of the second precision tier and the
mixed path's FP32 lane arithmetic) compiled for the host. Compares with numpy on the same
weighted systems; no GPU and no oracle involved."""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from tests._helpers import table1_cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_kernels", "mls_algebra.cu")


@pytest.fixture(scope="module")
def hk(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hk") / "libhk.so")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-shared",
                    "-Xcompiler", "-fPIC", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2510_18838_gb300", "csrc"), SRC, "-o", out],
                   check=True)
    L = ctypes.CDLL(out)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.hk_mls.restype = I
    L.hk_mls.argtypes = [I, I, I, I, I, P, P, D, D, D, P, P, I, P]
    L.hk_mls_f32.restype = I
    L.hk_mls_f32.argtypes = [I, I, I, I, I, P, P, ctypes.c_float, D, D, P, P, I]
    L.hk_recentre_basis.restype = None
    L.hk_recentre_basis.argtypes = [I, P, P]
    L.hk_solve_refined.restype = I
    L.hk_solve_refined.argtypes = [I, I, I, I, I, P, P, P, D, P, P, P, P]
    L.hk_recentre_from.restype = None
    L.hk_recentre_from.argtypes = [I, P, P, P]
    L.hk_mono.restype = I
    L.hk_mono.argtypes = [I, I, P]
    L.hk_mono_prod.restype = I
    L.hk_mono_prod.argtypes = [I, I, I]
    L.hk_weight.restype = D
    L.hk_weight.argtypes = [I, D]
    L.hk_pair_plan.restype = I
    L.hk_pair_plan.argtypes = [I, I, P, P, P]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def exps(hk, dim, count):
    out = []
    e = np.zeros(3, np.int32)
    for p in range(count):
        hk.hk_mono(dim, p, _p(e))
        out.append(tuple(e[:dim]))
    return out


def test_monomial_order_is_graded_lex(hk):
    assert exps(hk, 2, 6) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    assert exps(hk, 3, 10) == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0),
                               (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for dim, nm in ((2, 15), (3, 35)):
        ex = exps(hk, dim, nm)
        assert len(set(ex)) == nm and all(sum(e) <= 4 for e in ex)
        degs = [sum(e) for e in ex]
        assert degs == sorted(degs)
        for k, l in itertools.product(range(6 if dim == 2 else 10), repeat=2):
            prod = tuple(a + b for a, b in zip(ex[k], ex[l]))
            assert ex[hk.hk_mono_prod(dim, k, l)] == prod


@pytest.mark.parametrize("kind,q,expect", table1_cases())
def test_weight_values_of_table1(hk, kind, q, expect):
    """The library's weight function (compiled for the host in FP64) at the closed-form
    points of Table 1, the same fixture the oracle's weights are pinned to."""
    from paper_2510_18838_gb300.pcms import WEIGHTS
    assert hk.hk_weight(WEIGHTS[kind], q) == pytest.approx(expect, rel=1e-15, abs=1e-300)


def _system(dim, deg, n, seed):
    rng = np.random.default_rng(seed)
    r = 0.05
    u = rng.uniform(-1, 1, (n * 3, dim))
    u = u[np.linalg.norm(u, axis=1) < 0.999][:n]
    dx = np.zeros((len(u), 3))
    dx[:, :dim] = u * r
    q = np.linalg.norm(u, axis=1)
    w = (1 - q) ** 4 * (4 * q + 1)
    # graded-lex: by degree, then exponents descending lexicographically
    ex = sorted((e for e in itertools.product(range(deg + 1), repeat=dim) if sum(e) <= deg),
                key=lambda e: (sum(e), tuple(-x for x in e)))
    A = np.stack([np.prod(u ** np.array(e), axis=1) for e in ex], axis=1)
    return dx, u, w, A, r


@pytest.mark.parametrize("dim,deg", [(2, 0), (2, 1), (2, 2), (3, 1), (3, 2)])
def test_operator_weights_match_numpy(hk, dim, deg):
    dx, u, w, A, r = _system(dim, deg, 60, 10 * dim + deg)
    m = A.shape[1]
    nm = len([e for e in itertools.product(range(2 * deg + 1), repeat=dim) if sum(e) <= 2 * deg])
    mom = np.zeros(nm)
    out = np.zeros(m + 5)
    ok = hk.hk_mls(dim, deg, 0, 0, len(dx), _p(np.ascontiguousarray(dx)), None, 1.0 / r, 0.0,
                   1e-14, _p(mom), _p(out), 0, None)
    assert ok == 1
    y, amp = out[:m], out[m]
    G = (A * w[:, None]).T @ A
    y_ref = np.linalg.solve(G, np.eye(m)[0])
    np.testing.assert_allclose(y, y_ref, rtol=1e-10, atol=1e-12 * np.abs(y_ref).max())
    amp_ref = np.sqrt(G[0, 0]) * np.sum(np.abs(y_ref) * np.sqrt(np.diag(G)))
    assert amp == pytest.approx(amp_ref, rel=1e-10)
    assert amp >= 1.0 - 1e-12          # amp >= G_00 * y_0 = G_00 (G^-1)_00 >= 1
    # the shape functions w a^T y reproduce every basis monomial (moment conditions)
    N = w * (A @ y)
    np.testing.assert_allclose(N @ A, np.eye(m)[0], atol=1e-12)


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 2)])
@pytest.mark.parametrize("lam", [0.0, 0.25])
def test_one_shot_value_matches_weighted_lstsq(hk, dim, deg, lam):
    dx, u, w, A, r = _system(dim, deg, 80, 100 + 10 * dim + deg)
    m = A.shape[1]
    b = np.cos(7 * u[:, 0]) + u[:, -1] ** 2
    nm = len([e for e in itertools.product(range(2 * deg + 1), repeat=dim) if sum(e) <= 2 * deg])
    mom = np.zeros(nm + m)
    c0 = np.zeros(m + 5)
    ok = hk.hk_mls(dim, deg, 1, 0, len(dx), _p(np.ascontiguousarray(dx)), _p(b), 1.0 / r, lam,
                   1e-14, _p(mom), _p(c0), 0, None)
    assert ok == 1
    sw = np.sqrt(w)
    Aa = np.vstack([sw[:, None] * A, np.sqrt(lam) * np.eye(m)])
    ba = np.concatenate([sw * b, np.zeros(m)])
    c, *_ = np.linalg.lstsq(Aa, ba, rcond=None)
    assert c0[0] == pytest.approx(c[0], rel=1e-11, abs=1e-12)


def test_guard_flags_collinear_points(hk):
    t = np.linspace(-0.9, 0.9, 30)
    dx = np.zeros((30, 3))
    dx[:, 0] = 0.05 * t
    dx[:, 1] = 0.05 * 0.5 * t
    mom = np.zeros(15)
    y = np.zeros(11)
    for deg, ok in ((1, 0), (2, 0), (0, 1)):
        for rc in (0, 1):
            assert hk.hk_mls(2, deg, 0, 0, 30, _p(dx), None, 20.0, 0.0, 1e-14, _p(mom), _p(y),
                             rc, None) == ok


def _lopsided(dim, deg, n, seed, centre=0.62, spread=0.12):
    """A far target's neighbourhood: the selected sources lie in a blob on one side of the
    target (offsets in units of r around (centre, 0.3 centre, ..), spread `spread`), as after
    the radius doubling at the edge of a source cluster."""
    rng = np.random.default_rng(seed)
    r = 0.05
    c = np.zeros(dim)
    c[0], c[1] = centre, 0.3 * centre
    u = c + spread * rng.standard_normal((n * 3, dim))
    u = u[np.linalg.norm(u, axis=1) < 0.999][:n]
    dx = np.zeros((len(u), 3))
    dx[:, :dim] = u * r
    q = np.linalg.norm(u, axis=1)
    w = (1 - q) ** 4 * (4 * q + 1)
    ex = sorted((e for e in itertools.product(range(deg + 1), repeat=dim) if sum(e) <= deg),
                key=lambda e: (sum(e), tuple(-x for x in e)))
    A = np.stack([np.prod(u ** np.array(e), axis=1) for e in ex], axis=1)
    return dx, u, w, A, r


def _n_moments(dim, deg):
    return len([e for e in itertools.product(range(2 * deg + 1), repeat=dim) if sum(e) <= 2 * deg])


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 2)])
def test_recentred_basis_gives_the_same_fit(hk, dim, deg):
    """At lambda = 0 the fitted value does not depend on the polynomial basis: the second
    tier's re-centred, re-scaled basis must give the target-centred weighted least-squares
    value and the same operator row, while its amplification factor is much smaller."""
    dx, u, w, A, r = _lopsided(dim, deg, 400, 7 + dim + deg)
    m = A.shape[1]
    nm = _n_moments(dim, deg)
    b = np.cos(3 * u[:, 0]) + u[:, 1] ** 2
    dxc = np.ascontiguousarray(dx)
    sw = np.sqrt(w)
    c, *_ = np.linalg.lstsq(sw[:, None] * A, sw * b, rcond=None)
    out0, out1 = np.zeros(m + 5), np.zeros(m + 5)
    mom = np.zeros(nm + m)
    assert hk.hk_mls(dim, deg, 1, 0, len(dx), _p(dxc), _p(b), 1.0 / r, 0.0, 1e-14, _p(mom),
                     _p(out0), 0, None) == 1
    assert hk.hk_mls(dim, deg, 1, 0, len(dx), _p(dxc), _p(b), 1.0 / r, 0.0, 1e-14, _p(mom),
                     _p(out1), 1, None) == 1
    assert out1[0] == pytest.approx(c[0], rel=1e-9, abs=1e-12)
    assert out0[0] == pytest.approx(c[0], rel=1e-9, abs=1e-12)
    bas = out1[m + 1:m + 5]
    assert not np.allclose(bas, [0, 0, 0, 1])          # the basis did move
    assert out1[m] < out0[m] / 4                        # and the amplification dropped
    # operator rows N_j = w_j a(u'_j)^T y' equal the target-centred ones
    G = (A * w[:, None]).T @ A
    N_ref = w * (A @ np.linalg.solve(G, np.eye(m)[0]))
    rows = np.zeros(len(dx))
    out = np.zeros(m + 5)
    assert hk.hk_mls(dim, deg, 0, 0, len(dx), _p(dxc), None, 1.0 / r, 0.0, 1e-14, _p(mom[:nm]),
                     _p(out), 1, _p(rows)) == 1
    np.testing.assert_allclose(rows, N_ref, rtol=1e-8, atol=1e-10 * np.abs(N_ref).max())
    np.testing.assert_allclose(rows @ A, np.eye(m)[0], atol=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_recentre_basis_is_weighted_centroid_and_spread(hk, dim):
    dx, u, w, A, r = _lopsided(dim, 2, 300, 40 + dim)
    nm = _n_moments(dim, 2)
    mom = np.zeros(nm + 10)
    out = np.zeros(15)
    hk.hk_mls(dim, 2, 0, 0, len(dx), _p(np.ascontiguousarray(dx)), None, 1.0 / r, 0.0, 1e-14,
              _p(mom), _p(out), 0, None)
    got = np.zeros(4, np.float32)
    hk.hk_recentre_basis(dim, _p(mom), _p(got))
    c = (w[:, None] * u).sum(0) / w.sum()
    s = np.sqrt((w * ((u - c) ** 2).sum(1)).sum() / (dim * w.sum()))
    np.testing.assert_allclose(got[:dim], c, rtol=1e-6, atol=1e-7)
    assert got[3] == pytest.approx(1.0 / s, rel=1e-6)
    # zero spread (all neighbours at one point): no re-centring
    one = np.zeros(nm)
    one[0] = 2.0
    hk.hk_recentre_basis(dim, _p(one), _p(got))
    assert list(got) == [0.0, 0.0, 0.0, 1.0]


@pytest.mark.parametrize("dim", [2, 3])
def test_recentre_from_an_estimated_basis(hk, dim):
    """Tier 1 may assemble in an estimated basis b = (c_b, 1/s_b); the basis handed on to
    tier 2 is then the weighted centroid and spread of the neighbours in the original
    offsets, composed from the moments in b. From the identity it is recentre_basis
    bit for bit."""
    dx, u, w, A, r = _lopsided(dim, 2, 300, 60 + dim)
    nm = _n_moments(dim, 2)
    mom = np.zeros(nm + 10)
    out = np.zeros(15)
    hk.hk_mls(dim, 2, 0, 0, len(dx), _p(np.ascontiguousarray(dx)), None, 1.0 / r, 0.0, 1e-14,
              _p(mom), _p(out), 0, None)
    ident = np.array([0, 0, 0, 1], np.float32)
    a = np.zeros(4, np.float32)
    b = np.zeros(4, np.float32)
    hk.hk_recentre_basis(dim, _p(mom), _p(a))
    hk.hk_recentre_from(dim, _p(ident), _p(mom), _p(b))
    assert np.array_equal(a, b)
    # moments of the same neighbours in a rough estimate of the basis
    c = (w[:, None] * u).sum(0) / w.sum()
    s = np.sqrt((w * ((u - c) ** 2).sum(1)).sum() / (dim * w.sum()))
    est = np.zeros(4, np.float32)
    est[:dim] = (c + 0.07 * np.arange(1, dim + 1)).astype(np.float32)
    est[3] = np.float32(1.0 / (1.6 * s))
    up = (u - est[:dim].astype(np.float64)) * np.float64(est[3])
    exps_ = [e for e in itertools.product(range(5), repeat=dim) if sum(e) <= 4]
    exps_.sort(key=lambda e: (sum(e), tuple(-x for x in e)))
    mom_b = np.array([(w * np.prod(up ** np.array(e), axis=1)).sum() for e in exps_])
    assert len(mom_b) == nm
    got = np.zeros(4, np.float32)
    hk.hk_recentre_from(dim, _p(est), _p(mom_b), _p(got))
    np.testing.assert_allclose(got[:dim], c, rtol=1e-5, atol=1e-6)
    assert got[3] == pytest.approx(1.0 / s, rel=1e-5)
    # a degenerate spread in b keeps b
    one = np.zeros(nm)
    one[0] = 2.0
    hk.hk_recentre_from(dim, _p(est), _p(one), _p(got))
    assert np.array_equal(got, est)


def _gram(dim, deg, mom):
    """The moment matrix G_kl = mom[index of monomial k * monomial l] (graded-lex order)."""
    ex = sorted((e for e in itertools.product(range(2 * deg + 1), repeat=dim) if sum(e) <= 2 * deg),
                key=lambda e: (sum(e), tuple(-x for x in e)))
    basis = [e for e in ex if sum(e) <= deg]
    idx = {e: i for i, e in enumerate(ex)}
    return np.array([[mom[idx[tuple(np.add(a, b))]] for b in basis] for a in basis])


def _refined(hk, dim, deg, fused, pairs, mom, at=None, amp_accept=1e30):
    m = mono = len([e for e in itertools.product(range(deg + 1), repeat=dim) if sum(e) <= deg])
    nm = _n_moments(dim, deg)
    nacc = nm + m if fused else nm
    hi = np.asarray(mom[:nacc], np.float64).astype(np.float32)
    lo = (np.asarray(mom[:nacc]) - hi.astype(np.float64)).astype(np.float32) if pairs \
        else np.zeros(nacc, np.float32)
    yh, yl = np.zeros(m, np.float32), np.zeros(m, np.float32)
    c0, amp = np.zeros(1), np.zeros(1)
    atp = None if at is None else _p(np.ascontiguousarray(at, np.float64))
    rc = hk.hk_solve_refined(dim, deg, fused, pairs, nacc, _p(hi), _p(lo), atp,
                             float(amp_accept), _p(yh), _p(yl), _p(c0), _p(amp))
    stored = hi.astype(np.float64) + lo.astype(np.float64)
    return rc, yh.astype(np.float64) + yl.astype(np.float64), c0[0], amp[0], stored


@pytest.mark.parametrize("dim,deg,fused,pairs",
                         [(2, 2, 1, 1), (2, 2, 0, 0), (3, 2, 0, 0), (3, 2, 1, 1), (2, 1, 0, 0),
                          (3, 1, 1, 0), (2, 1, 1, 1)])
def test_refined_fp32_solve_reaches_the_exact_solution(hk, dim, deg, fused, pairs):
    """The mixed tiers solve the stored FP32 moments with an FP32 factorization and
    double-FP32 refinement. On well-spread neighbourhoods y must reach the exact solution of
    that FP32-valued system to 2^-20 / amp relative (what moves c_0 by at most 2^-20 of the
    field; an FP32 solve alone is ~kappa 2^-24 off), c_0 likewise, amp the exact one's to
    FP32 rounding. With amp above the caller's acceptance bound it stops after the FP32 solve
    and reports amp (code 2)."""
    dx, u, w, A, r = _system(dim, deg, 400, 90 + 7 * dim + deg + pairs)
    m = A.shape[1]
    nm = _n_moments(dim, deg)
    b = np.cos(3 * u[:, 0]) + u[:, 1] ** 2
    mom = np.zeros(nm + m)
    out = np.zeros(m + 5)
    hk.hk_mls(dim, deg, 1, 0, len(dx), _p(np.ascontiguousarray(dx)), _p(b), 1.0 / r, 0.0,
              1e-14, _p(mom), _p(out), 0, None)
    rc, y, c0, amp, stored = _refined(hk, dim, deg, fused, pairs, mom)
    assert rc == 1
    G = _gram(dim, deg, stored[:nm])
    y_ex = np.linalg.solve(G, np.eye(m)[0])
    d = np.sqrt(np.diag(G))
    amp_ex = d[0] * np.sum(np.abs(y_ex) * d)
    assert amp == pytest.approx(amp_ex, rel=1e-5)
    assert np.abs(y - y_ex).max() <= 2.0 ** -20 / max(amp_ex, 1.0) * np.abs(y_ex).max()
    y32 = np.linalg.solve(G.astype(np.float32), np.eye(m, dtype=np.float32)[0]).astype(np.float64)
    assert np.abs(y - y_ex).max() < np.abs(y32 - y_ex).max()        # better than FP32 alone
    if fused:
        assert c0 == pytest.approx(y_ex @ stored[nm:nm + m], rel=2e-6, abs=1e-12)
    rc2, _, _, amp2, _ = _refined(hk, dim, deg, fused, pairs, mom, amp_accept=amp_ex / 2)
    assert rc2 == 2 and amp2 == pytest.approx(amp_ex, rel=1e-3)


@pytest.mark.parametrize("dim", [2, 3])
def test_refined_fp32_solve_in_a_recentred_basis(hk, dim):
    """A one-sided neighbourhood: in the target-centred basis amp is large and the refined
    solve may decline (the FP64 solve then runs); in the re-centred basis, with a_t = a(-c/s),
    it converges and c_0 is the weighted least-squares value."""
    dx, u, w, A, r = _lopsided(dim, 2, 400, 70 + dim)
    m = A.shape[1]
    nm = _n_moments(dim, 2)
    b = np.cos(3 * u[:, 0]) + u[:, 1] ** 2
    sw = np.sqrt(w)
    c_ls, *_ = np.linalg.lstsq(sw[:, None] * A, sw * b, rcond=None)
    mom = np.zeros(nm + m)
    out = np.zeros(m + 5)
    hk.hk_mls(dim, 2, 1, 0, len(dx), _p(np.ascontiguousarray(dx)), _p(b), 1.0 / r, 0.0, 1e-14,
              _p(mom), _p(out), 0, None)
    rc, y, c0, amp, _ = _refined(hk, dim, 2, 1, 1, mom)
    assert rc in (0, 1)
    if rc == 1:
        assert c0 == pytest.approx(c_ls[0], rel=1e-6)
    bas = np.zeros(4, np.float32)
    hk.hk_recentre_basis(dim, _p(mom), _p(bas))
    c, ws = bas[:dim].astype(np.float64), np.float64(bas[3])
    up = (u - c) * ws
    ex = sorted((e for e in itertools.product(range(5), repeat=dim) if sum(e) <= 4),
                key=lambda e: (sum(e), tuple(-x for x in e)))
    ex2 = [e for e in ex if sum(e) <= 2]
    mom_c = np.array([(w * np.prod(up ** np.array(e), axis=1)).sum() for e in ex] +
                     [(w * b * np.prod(up ** np.array(e), axis=1)).sum() for e in ex2])
    at = np.array([np.prod((-c * ws) ** np.array(e)) for e in ex2])
    rc, y, c0, amp_c, _ = _refined(hk, dim, 2, 1, 1, mom_c, at=at)
    assert rc == 1
    assert c0 == pytest.approx(c_ls[0], rel=1e-7)
    assert amp_c < out[m] / 4


def test_refined_fp32_solve_hands_singular_systems_to_fp64(hk):
    """Collinear neighbours make a quadratic system singular: the refined FP32 solve must
    decline (the FP64 solve and its guard then decide), never return a value."""
    rng = np.random.default_rng(3)
    t = rng.uniform(-0.9, 0.9, 200)
    u = np.stack([t, 0.5 * t], 1)
    w = (1 - np.abs(t)) ** 4 * (4 * np.abs(t) + 1)
    ex = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3),
          (4, 0), (3, 1), (2, 2), (1, 3), (0, 4)]
    mom = np.array([(w * u[:, 0] ** a * u[:, 1] ** c).sum() for a, c in ex])
    rc, *_ = _refined(hk, 2, 2, 0, 0, mom)
    assert rc == 0


def _f32_case(kind_of, n, seed):
    if kind_of == "ball":
        dx, u, w, A, r = _system(2, 2, n, seed)
    else:
        dx, u, w, A, r = _lopsided(2, 2, n, seed)
    dx32 = dx.astype(np.float32)
    u64 = dx32[:, :2].astype(np.float64) / np.float64(np.float32(r))
    b32 = (np.cos(3 * u64[:, 0]) * np.sin(2 * u64[:, 1]) + 0.5).astype(np.float32)
    # the exact fit of the FP32 data (the values the mixed path receives)
    inv_r = np.float32(1.0 / r)
    u = dx32[:, :2].astype(np.float64) * np.float64(inv_r)
    q = np.linalg.norm(u, axis=1)
    w = (1 - q) ** 4 * (4 * q + 1)
    ex = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    A = np.stack([u[:, 0] ** a * u[:, 1] ** c for a, c in ex], axis=1)
    sw = np.sqrt(w)
    c, *_ = np.linalg.lstsq(sw[:, None] * A, sw * b32.astype(np.float64), rcond=None)
    return np.ascontiguousarray(dx32), b32, inv_r, c[0]


@pytest.mark.parametrize("case,n", [("ball", 20000), ("lopsided", 20000), ("lopsided", 3000)])
def test_fp32_blocked_compensation_error_model(hk, case, n):
    """The mixed path's FP32 lane arithmetic (32 lanes) against the exact fit of the same FP32
    data: blocked compensation stays within the bound the tier routing relies on
    (|err| <= 3.4 amp 2^-24 / sqrt(n), checked with a factor 2), and beats plain sums."""
    dx32, b32, inv_r, ref = _f32_case(case, n, 900 + n)
    nn = len(dx32)
    res = {}
    for scheme in (0, 1):
        out = np.zeros(2)
        assert hk.hk_mls_f32(2, 2, scheme, 0, nn, _p(dx32), _p(b32), float(inv_r), 0.0, 1e-14,
                             None, _p(out), 32) == 1
        res[scheme] = (abs(out[0] - ref), out[1])
    err_bk, amp = res[1]
    assert err_bk <= 2 * 3.4 * amp * 2.0 ** -24 / np.sqrt(nn)
    assert err_bk < res[0][0] / 4


def test_fp32_recentred_tier_accuracy(hk):
    """The second tier: blocked compensation in the re-centred basis of a lopsided
    neighbourhood is within the error model with the (smaller) re-centred amplification."""
    dx32, b32, inv_r, ref = _f32_case("lopsided", 8000, 77)
    nn = len(dx32)
    # basis from the target-centred FP64 moments, as k_solve derives it
    nm = _n_moments(2, 2)
    mom = np.zeros(nm + 6)
    out = np.zeros(11)
    hk.hk_mls(2, 2, 0, 0, nn, _p(dx32.astype(np.float64)), None, float(inv_r), 0.0, 1e-14,
              _p(mom), _p(out), 0, None)
    amp_tc = out[6]
    bas = np.zeros(4, np.float32)
    hk.hk_recentre_basis(2, _p(mom), _p(bas))
    res = np.zeros(2)
    assert hk.hk_mls_f32(2, 2, 1, 0, nn, _p(dx32), _p(b32), float(inv_r), 0.0, 1e-14, _p(bas),
                         _p(res), 32) == 1
    err, amp_rc = abs(res[0] - ref), res[1]
    assert amp_rc < amp_tc / 10
    assert err <= 2 * 3.4 * amp_rc * 2.0 ** -24 / np.sqrt(nn)


@pytest.mark.parametrize("t", [(-0.2, -0.2, -0.2), (-0.25, -0.25, 0.2), (-0.3, -0.1, 0.5)])
def test_fp64_refine_pass_on_extrapolating_targets(hk, t):
    """The FP64 path's refine pass. A 3D quadratic fit at a target outside the sources
    reproduces a quadratic field exactly in exact arithmetic, so the error of c_0 is pure
    rounding. In the target-centred basis amp is far above AMP_FP64 = 256 and the FP64
    normal equations lose digits (error ~ amp 2^-53, here up to 2e-10 of the field's size);
    the re-centred basis cuts amp and the error by a factor of more than 50, to below 1e-12."""
    rng = np.random.default_rng(5)
    src = rng.uniform(size=(3, 12000))
    tgt = np.array(t)
    r = 0.48
    d = src - tgt[:, None]
    sel = (d ** 2).sum(0) < r * r
    dx = np.ascontiguousarray(d[:, sel].T)
    s = src[:, sel]
    f = lambda x, y, z: 1.0 + 2.0 * x - y + 0.5 * z + x * x - 0.7 * x * y + 0.3 * z * z + y * z
    b = f(*s)
    exact = f(*tgt)
    scale = np.abs(b).max()
    n = len(b)
    res = {}
    for rc in (0, 1):
        mom = np.zeros(_n_moments(3, 2) + 10)
        out = np.zeros(16)
        assert hk.hk_mls(3, 2, 1, 0, n, _p(dx), _p(b), 1.0 / r, 0.0, 1e-14, _p(mom), _p(out),
                         rc, None) == 1
        res[rc] = (abs(out[0] - exact) / scale, out[10])
    (err_tc, amp_tc), (err_rc, amp_rc) = res[0], res[1]
    assert amp_tc > 256 * 100
    assert amp_rc < amp_tc / 50
    assert err_rc <= 1e-12
    assert err_rc < err_tc / 50


@pytest.mark.parametrize("dim,mdeg,expect", [(2, 2, 6), (2, 4, 16), (3, 2, 11), (3, 4, 33)])
def test_pairing_of_the_fp32_moment_terms(hk, dim, mdeg, expect):
    """The compile-time pairing of the FP32 moment terms for two-lane FP32 instructions. The
    scalar chain forms each term w u^e as its parent (e with its first positive exponent
    lowered by one) times u of that variable. A packed pair (p, q) is one two-lane product of
    the parent pair, so p and q must share that variable and their parents must be partners,
    p's parent in lane 0. Pairs hold terms of one degree; w (degree 0) is alone. The count of
    instructions for the terms and their sums (a packed pair: product + sum, or one fused
    multiply-add at the top degree; an unpacked pair: two products + one packed sum, or two
    fused multiply-adds at the top degree; a single: product + sum, or one fused multiply-add)
    is fixed per shape (the scalar chain takes 2 per term, 1 at the top degree)."""
    n = _n_moments(dim, mdeg // 2)
    partner = np.zeros(n, np.int32)
    first = np.zeros(n, np.int32)
    packed = np.zeros(n, np.int32)
    assert hk.hk_pair_plan(dim, mdeg, _p(partner), _p(first), _p(packed)) == n
    ex = exps(hk, dim, n)
    deg = [sum(e) for e in ex]
    index = {e: i for i, e in enumerate(ex)}

    def var(e):
        return next(d for d in range(dim) if e[d] > 0)

    def parent(e):
        v = var(e)
        return index[tuple(x - (d == v) for d, x in enumerate(e))]

    assert partner[0] == -1
    count = 1   # w into its sum
    for p in range(1, n):
        q = partner[p]
        top = deg[p] == mdeg
        if q < 0:
            assert not first[p] and not packed[p]
            count += 1 if top else 2
            continue
        assert partner[q] == p and q != p and deg[q] == deg[p]
        assert first[p] + first[q] == 1
        if not first[p]:
            assert not packed[p]
            continue
        if packed[p]:
            assert var(ex[p]) == var(ex[q])
            a, b = parent(ex[p]), parent(ex[q])
            assert partner[a] == b and first[a] == 1
            count += 1 if top else 2
        else:
            count += 2 if top else 3
    assert count == expect
    scalar = 1 + sum(1 if deg[p] == mdeg else 2 for p in range(1, n))
    assert count < scalar
