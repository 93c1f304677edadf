"""Seeded synthetic inputs shaped like the paper's field-transfer workloads.

This module only draws coordinates, meshes and field samples. It holds none of the
transfer method's arithmetic (no neighbour search, no weights, no fitting, no point
location), so both the CPU oracle and the CUDA path can be fed from it without sharing
any of the method's code.

All point arrays are structure-of-arrays, ``float64[dim, n]``, C-contiguous. Every
generator takes explicit seeds (``numpy.random.default_rng``, PCG64).

The paper's own workloads (the WEST, LTX and D3D meshes and fields of Sec. 3.2 and
Sec. 6) are not available; these generators stand in for them:

* ``mls_2d_small``     2D uniform clouds, 10,000 -> 10,000, field sin(2 pi x) cos(2 pi y).
* ``jittered_mesh``    512 x 512 structured grid split into 524,288 CCW triangles with
                       interior vertices moved inside a disk of radius 0.3 h.
* ``mls_2d_gaussian``  4M sources from a mixture of 8 clipped Gaussians, 4M uniform targets.
* ``mls_3d_slab``      8M sources (uniform cube plus a dense slab), 8M uniform targets,
                       16 random trigonometric fields of degree <= 4.
* ``request_stream``   Poisson stream of mixed MLS / mesh transfer requests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def uniform_points(n: int, dim: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` i.i.d. uniform points in ``[lo, hi]^dim`` as ``float64[dim, n]``."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(lo, hi, size=(n, dim))
    return np.ascontiguousarray(pts.T)


def sincos_field(pts: np.ndarray) -> np.ndarray:
    """f = sin(2 pi x) cos(2 pi y), evaluated in float64."""
    return np.sin(TWO_PI * pts[0]) * np.cos(TWO_PI * pts[1])


# ---------------------------------------------------------------------------------------
# 2D MLS, small: 10k -> 10k uniform, linear basis, Wendland C2, r = 0.03
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class MLSCase:
    src: np.ndarray          # float64[dim, ns]
    tgt: np.ndarray          # float64[dim, nt]
    fields: np.ndarray       # float64 or float32 [F, ns]
    degree: int
    radius: float
    min_neighbors: int = 0
    name: str = ""

    @property
    def dim(self) -> int:
        return self.src.shape[0]


def mls_2d_small(n_src: int = 10_000, n_tgt: int = 10_000, seed_src: int = 101,
                 seed_tgt: int = 102, radius: float = 0.03, degree: int = 1) -> MLSCase:
    src = uniform_points(n_src, 2, seed_src)
    tgt = uniform_points(n_tgt, 2, seed_tgt)
    f = sincos_field(src)[None, :].copy()
    return MLSCase(src, tgt, f, degree, radius, 0, "mls2d_uniform_10k_linear_r0.03_fp64")


# ---------------------------------------------------------------------------------------
# 2D mesh: 512 x 512 jittered grid, 524,288 triangles, 1M uniform targets
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class MeshCase:
    xy: np.ndarray           # float64[2, nv]
    tri: np.ndarray          # int32[3, nt], counter-clockwise
    field: np.ndarray        # float64[nv]
    pts: np.ndarray          # float64[2, q]
    name: str = ""


def jittered_grid_mesh(n: int = 512, jitter: float = 0.3, seed: int = 201):
    """Structured n x n grid on [0,1]^2, each cell split along its (i,j)-(i+1,j+1)
    diagonal. Interior vertices are moved uniformly inside a disk of radius jitter*h
    (boundary vertices stay put), so no triangle can invert (max displacement sum
    2*0.3h < 0.707h, the right triangle's altitude).

    Vertex (i, j) has index j*(n+1)+i. Cell (i, j) gives triangle 2*(j*n+i) (lower right:
    (i,j),(i+1,j),(i+1,j+1)) and 2*(j*n+i)+1 (upper left: (i,j),(i+1,j+1),(i,j+1)).
    Returns (xy float64[2, (n+1)^2], tri int32[3, 2 n^2]).
    """
    h = 1.0 / n
    idx = np.arange(n + 1, dtype=np.float64)
    gx, gy = np.meshgrid(idx * h, idx * h, indexing="xy")   # gx[j, i] = i*h
    x = gx.ravel().copy()
    y = gy.ravel().copy()
    if jitter > 0:
        rng = np.random.default_rng(seed)
        nv = (n + 1) * (n + 1)
        rad = jitter * h * np.sqrt(rng.uniform(0.0, 1.0, nv))
        ang = rng.uniform(0.0, TWO_PI, nv)
        ii = np.tile(np.arange(n + 1), n + 1)
        jj = np.repeat(np.arange(n + 1), n + 1)
        interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n)
        x[interior] += (rad * np.cos(ang))[interior]
        y[interior] += (rad * np.sin(ang))[interior]
    xy = np.stack([x, y])
    i = np.tile(np.arange(n), n)
    j = np.repeat(np.arange(n), n)
    v00 = j * (n + 1) + i
    v10 = v00 + 1
    v11 = v00 + (n + 1) + 1
    v01 = v00 + (n + 1)
    tri = np.empty((3, 2 * n * n), dtype=np.int32)
    tri[0, 0::2], tri[1, 0::2], tri[2, 0::2] = v00, v10, v11
    tri[0, 1::2], tri[1, 1::2], tri[2, 1::2] = v00, v11, v01
    return np.ascontiguousarray(xy), tri


def mesh_2d(n: int = 512, n_pts: int = 1_000_000, seed_mesh: int = 201,
            seed_pts: int = 202, jitter: float = 0.3) -> MeshCase:
    xy, tri = jittered_grid_mesh(n, jitter, seed_mesh)
    field = xy[0] ** 2 + 3.0 * xy[0] * xy[1]
    pts = uniform_points(n_pts, 2, seed_pts)
    return MeshCase(xy, tri, field, pts, f"mesh2d_{n}x{n}_jitter{jitter}_{n_pts}pts")


# ---------------------------------------------------------------------------------------
# 2D MLS at scale: 4M sources from 8 clipped Gaussians, 4M uniform targets, quadratic
# ---------------------------------------------------------------------------------------
def gaussian_mixture_points(n: int, seed_centres: int = 301, seed_pts: int = 302,
                            n_comp: int = 8) -> np.ndarray:
    """Equal-weight mixture of ``n_comp`` isotropic Gaussians with centres uniform in
    [0.1, 0.9]^2 and sigma_k = 0.02 * 5^(k/(n_comp-1)) (log-spaced 0.02 .. 0.1), clipped to
    the unit square by rejection (rejected draws are re-drawn from the same component)."""
    crng = np.random.default_rng(seed_centres)
    centres = crng.uniform(0.1, 0.9, size=(n_comp, 2))
    sig = 0.02 * 5.0 ** (np.arange(n_comp) / (n_comp - 1))
    rng = np.random.default_rng(seed_pts)
    comp = rng.integers(0, n_comp, size=n)
    pts = centres[comp] + sig[comp, None] * rng.standard_normal((n, 2))
    bad = np.nonzero(((pts < 0.0) | (pts > 1.0)).any(axis=1))[0]
    while bad.size:
        c = comp[bad]
        pts[bad] = centres[c] + sig[c, None] * rng.standard_normal((bad.size, 2))
        sub = ((pts[bad] < 0.0) | (pts[bad] > 1.0)).any(axis=1)
        bad = bad[sub]
    return np.ascontiguousarray(pts.T)


def mls_2d_gaussian(n_src: int = 4_000_000, n_tgt: int = 4_000_000, radius: float = 0.01,
                    degree: int = 2, min_neighbors: int = 10) -> MLSCase:
    src = gaussian_mixture_points(n_src)
    tgt = uniform_points(n_tgt, 2, 303)
    f = sincos_field(src)[None, :].copy()
    return MLSCase(src, tgt, f, degree, radius, min_neighbors,
                   f"mls2d_gauss8_{n_src}_quadratic_r{radius}_mixed")


# ---------------------------------------------------------------------------------------
# 3D MLS multi-field: 8M sources (uniform + dense slab), 8M targets, 16 fields
# ---------------------------------------------------------------------------------------
def slab_points(n: int, frac_slab: float = 0.2, seed: int = 401) -> np.ndarray:
    """(1-frac_slab) n uniform in [0,1]^3 plus frac_slab n uniform in [0,1]^2 x [0.45,0.55]."""
    rng = np.random.default_rng(seed)
    n_slab = int(round(frac_slab * n))
    a = rng.uniform(0.0, 1.0, size=(n - n_slab, 3))
    b = rng.uniform(0.0, 1.0, size=(n_slab, 3))
    b[:, 2] = 0.45 + 0.1 * b[:, 2]
    return np.ascontiguousarray(np.concatenate([a, b]).T)


def trig_fields(pts: np.ndarray, n_fields: int = 16, max_deg: int = 4,
                seed0: int = 410, chunk: int = 1 << 20) -> np.ndarray:
    """Random trigonometric polynomials f_k = sum_{p+q+s<=max_deg} a cos(2 pi (px+qy+sz))
    + b sin(2 pi (px+qy+sz)), coefficients N(0,1)/sqrt(#terms) drawn with seed seed0+k.
    Evaluated in float64 (complex exponentials), returned as float32[n_fields, n]."""
    dim = pts.shape[0]
    terms = [t for t in np.ndindex(*([max_deg + 1] * dim)) if sum(t) <= max_deg]
    nt = len(terms)
    coef = np.empty((n_fields, 2 * nt))
    for k in range(n_fields):
        r = np.random.default_rng(seed0 + k)
        coef[k] = r.standard_normal(2 * nt) / math.sqrt(nt)
    n = pts.shape[1]
    out = np.empty((n_fields, n), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        ph = [np.exp(1j * TWO_PI * pts[d, s:e]) for d in range(dim)]
        pw = [[np.ones(e - s, dtype=np.complex128)] for _ in range(dim)]
        for d in range(dim):
            for _ in range(max_deg):
                pw[d].append(pw[d][-1] * ph[d])
        basis = np.empty((2 * nt, e - s))
        for t_i, t in enumerate(terms):
            z = pw[0][t[0]]
            for d in range(1, dim):
                z = z * pw[d][t[d]]
            basis[2 * t_i] = z.real
            basis[2 * t_i + 1] = z.imag
        out[:, s:e] = (coef @ basis).astype(np.float32)
    return out


def mls_3d_slab(n_src: int = 8_000_000, n_tgt: int = 8_000_000, radius: float = 0.012,
                degree: int = 2, n_fields: int = 16) -> MLSCase:
    src = slab_points(n_src)
    tgt = uniform_points(n_tgt, 3, 402)
    f = trig_fields(src, n_fields)
    return MLSCase(src, tgt, f, degree, radius, 0,
                   f"mls3d_slab_{n_src}_quadratic_r{radius}_{n_fields}fields_mixed")


# ---------------------------------------------------------------------------------------
# 5D distribution function (stand-in for the paper's GNET energetic-particle distribution)
# ---------------------------------------------------------------------------------------
def slowing_down_points(n: int, seed: int, vc: float = 0.3) -> np.ndarray:
    """float64 [5, n] phase-space points (x, y, z, v_par, v_perp): positions uniform in the
    unit cube; speeds v in (0, 1] from the classical slowing-down shape, density in 3D velocity
    space ~ 1 / (v^3 + vc^3), i.e. speed density ~ v^2 / (v^3 + vc^3), with CDF
    F(v) = ln(1 + v^3/vc^3) / ln(1 + 1/vc^3), sampled by inversion:
    v = vc (exp(u ln(1 + 1/vc^3)) - 1)^(1/3); the pitch xi is uniform in [-1, 1] (isotropic):
    v_par = v xi, v_perp = v sqrt(1 - xi^2)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(3, n))
    u = rng.uniform(0.0, 1.0, size=n)
    v = np.cbrt(vc ** 3 * np.expm1(u * np.log1p(1.0 / vc ** 3)))
    xi = rng.uniform(-1.0, 1.0, size=n)
    vel = np.stack([v * xi, v * np.sqrt(1.0 - xi * xi)])
    return np.ascontiguousarray(np.concatenate([pos, vel]))


def distribution_5d_field(pts: np.ndarray, vc: float = 0.3) -> np.ndarray:
    """A smooth 5D distribution value: a Gaussian radial profile times a slowing-down speed
    factor 1 / (v^3 + vc^3) and a mild pitch anisotropy."""
    x, y, z, vpar, vperp = pts
    v2 = vpar * vpar + vperp * vperp
    radial = np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.08) * (1.0 + 0.3 * np.cos(2 * np.pi * z))
    return radial / (v2 * np.sqrt(v2) + vc ** 3) * (1.0 + 0.2 * vpar / np.sqrt(v2 + 1e-12))


def mls_5d_distribution(n_src: int = 400_000, n_tgt: int = 200_000, radius: float = 0.17,
                        degree: int = 2, min_neighbors: int = 30) -> MLSCase:
    src = slowing_down_points(n_src, 501)
    tgt = slowing_down_points(n_tgt, 502)
    f = distribution_5d_field(src)[None, :].copy()
    return MLSCase(src, tgt, f, degree, radius, min_neighbors,
                   f"mls5d_slowing_down_{n_src}_to_{n_tgt}_quadratic_r{radius}_fp64")


# ---------------------------------------------------------------------------------------
# Serving: Poisson stream of mixed transfer requests
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class Request:
    rid: int
    kind: str               # "mls" or "mesh"
    arrival_s: float        # offset from stream start
    dim: int
    degree: int
    n_src: int              # MLS: sources; mesh: triangles per side^2 * 2 (see mesh_n)
    n_tgt: int
    n_fields: int
    radius: float
    reuse_of: int           # -1, or the rid of an earlier MLS request whose map it reuses
    mesh_n: int = 0         # mesh: cells per side
    seed: int = 0


def request_stream(n_req: int = 2000, seed: int = 501, rate_hz: float = 2000.0,
                   pts_lo: float = 1e3, pts_hi: float = 2e6, reuse_frac: float = 0.3,
                   mesh_frac: float = 0.5, max_pts: int | None = None) -> list[Request]:
    """Request descriptors only (no arrays). Point counts are log-uniform in
    [pts_lo, pts_hi]; MLS radius gives k neighbours on average, k log-uniform in
    [max(10, 2m), 300]; mesh requests are 2D jittered grids with T log-uniform in
    [2e3, 2e6]; reuse_frac of the MLS requests reuse an earlier MLS request's map
    (same geometry, new field values)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_req))
    out: list[Request] = []
    mls_ids: list[int] = []
    hi = pts_hi if max_pts is None else min(pts_hi, max_pts)
    for i in range(n_req):
        u = rng.uniform(size=8)
        is_mesh = u[0] < mesh_frac
        n_tgt = int(math.exp(math.log(pts_lo) + u[1] * (math.log(hi) - math.log(pts_lo))))
        n_fields = int(rng.integers(1, 17))
        if is_mesh:
            n_tri = math.exp(math.log(2e3) + u[2] * (math.log(hi) - math.log(2e3)))
            mesh_n = max(8, int(round(math.sqrt(n_tri / 2.0))))
            out.append(Request(i, "mesh", float(t[i]), 2, 1, 2 * mesh_n * mesh_n, n_tgt,
                               1, 0.0, -1, mesh_n, seed * 100_000 + i))
            continue
        if mls_ids and u[3] < reuse_frac:
            src_req = out[mls_ids[int(rng.integers(0, len(mls_ids)))]]
            root = src_req.reuse_of if src_req.reuse_of >= 0 else src_req.rid
            out.append(dataclasses.replace(src_req, rid=i, arrival_s=float(t[i]),
                                           n_fields=n_fields, reuse_of=root))
            mls_ids.append(i)
            continue
        dim = 2 if u[4] < 0.5 else 3
        degree = 1 if u[5] < 0.5 else 2
        m = math.comb(dim + degree, degree)
        n_src = int(math.exp(math.log(pts_lo) + u[6] * (math.log(hi) - math.log(pts_lo))))
        k_lo = max(10.0, 2.0 * m)
        k = math.exp(math.log(k_lo) + u[7] * (math.log(300.0) - math.log(k_lo)))
        c_d = math.pi if dim == 2 else 4.0 * math.pi / 3.0
        radius = (k / (c_d * n_src)) ** (1.0 / dim)
        out.append(Request(i, "mls", float(t[i]), dim, degree, n_src, n_tgt, n_fields,
                           radius, -1, 0, seed * 100_000 + i))
        mls_ids.append(i)
    return out


def request_arrays(req: Request):
    """Materialise one request's inputs (host numpy). MLS: (src, tgt, fields float32[F,ns]);
    mesh: (xy, tri, nodal field, pts). A reused MLS request draws the same geometry as
    the request it reuses (same seed) and new field values."""
    if req.kind == "mesh":
        xy, tri = jittered_grid_mesh(req.mesh_n, 0.3, req.seed)
        field = xy[0] ** 2 + 3.0 * xy[0] * xy[1]
        pts = uniform_points(req.n_tgt, 2, req.seed + 1)
        return xy, tri, field, pts
    src = uniform_points(req.n_src, req.dim, req.seed)
    tgt = uniform_points(req.n_tgt, req.dim, req.seed + 1)
    fields = trig_fields(src, req.n_fields, max_deg=2, seed0=1000 + 37 * req.rid)
    return src, tgt, fields
