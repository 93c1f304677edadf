"""CPU check of the CUDA library's per-target MLS algebra (moment accumulation, monomial
tables, guarded LDL^T solve) compiled for the host. Compares with numpy on the same
weighted systems; no GPU and no oracle involved."""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

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
    L.hk_mls.argtypes = [I, I, I, I, I, P, P, D, D, D, P, P]
    L.hk_mono.restype = I
    L.hk_mono.argtypes = [I, I, P]
    L.hk_mono_prod.restype = I
    L.hk_mono_prod.argtypes = [I, I, I]
    L.hk_weight.restype = D
    L.hk_weight.argtypes = [I, D]
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


def test_wendland_value(hk):
    for q, v in [(0.0, 1.0), (0.5, 0.1875), (0.25, 0.6328125)]:
        assert hk.hk_weight(0, q) == pytest.approx(v, rel=1e-15)


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
    out = np.zeros(m + 1)
    ok = hk.hk_mls(dim, deg, 0, 0, len(dx), _p(np.ascontiguousarray(dx)), None, 1.0 / r, 0.0,
                   1e-14, _p(mom), _p(out))
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
    c0 = np.zeros(m + 1)
    ok = hk.hk_mls(dim, deg, 1, 0, len(dx), _p(np.ascontiguousarray(dx)), _p(b), 1.0 / r, lam,
                   1e-14, _p(mom), _p(c0))
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
    y = np.zeros(7)
    assert hk.hk_mls(2, 1, 0, 0, 30, _p(dx), None, 20.0, 0.0, 1e-14, _p(mom), _p(y)) == 0
    assert hk.hk_mls(2, 2, 0, 0, 30, _p(dx), None, 20.0, 0.0, 1e-14, _p(mom), _p(y)) == 0
    assert hk.hk_mls(2, 0, 0, 0, 30, _p(dx), None, 20.0, 0.0, 1e-14, _p(mom), _p(y)) == 1
