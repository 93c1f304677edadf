// projection.cu -- conservative L2 projection of a piecewise-linear (P1) field from one 2D
// triangle mesh to another through their intersection (Sec. 3.2.2, mesh intersection).
//
// With N_A the target's P1 shape functions, the projected field f_t solves M f_t = b with
// the consistent mass matrix M_AB = integral of N_A N_B and b_A = integral of N_A f_s. The
// integrand of b is smooth only on the pieces where one source and one target triangle
// overlap, so b is integrated over that supermesh:
//   1. k_supermesh_rhs, one thread per target triangle T: the source triangles listed in the
//      source mesh's grid cells under T's bounding box are the candidates; a pair whose
//      boxes overlap is taken once, in the cell of the lower-left corner of the boxes'
//      intersection. Each candidate S is clipped to T (Sutherland-Hodgman against T's three
//      edges, at most six vertices), the polygon is split into a fan and each sub-triangle is
//      integrated with the edge-midpoint rule, exact for the product of two linear functions.
//      The thread keeps T's three contributions and the pieces' area in registers.
//   2. k_vertex_gather: b_A = the sum over the triangles at vertex A, in triangle order (a
//      vertex-to-triangle list built once per mesh), so the result does not depend on the
//      order in which threads finish.
//   3. M f = b by conjugate gradients with a Jacobi preconditioner, M applied without
//      storing it: (M x)_A = sum over triangles T at A of |T|/12 (x_A + x_a + x_b + x_c).
//      Dot products are two-level fixed-order sums and the step sizes stay on the device; the
//      residual is read back every CG_CHECK iterations.
// Everything is FP64: the geometry decides which pieces exist, and the solve is short (the
// Jacobi-scaled P1 mass matrix has a condition number of a few units).
#include <algorithm>
#include <cmath>

#include "pcms_internal.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

constexpr int PJ_THREADS = 256;
constexpr int PJ_BLOCKS = 1024;   // partial sums of the dot products (fixed, for a fixed order)
constexpr int CG_CHECK = 8;

int pj_blocks(int64_t n) {
    const int64_t need = (n + PJ_THREADS - 1) / PJ_THREADS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 16));
}

// the cell of the source mesh's grid that holds coordinate x (clamped), as in its binning
__device__ __forceinline__ int grid_cell(double x, double lo, double inv_h, int n) {
    double f = floor((x - lo) * inv_h);
    f = fmin(fmax(f, 0.0), (double)(n - 1));
    return (int)f;
}

__device__ __forceinline__ double orient2(double ax, double ay, double bx, double by, double px,
                                          double py) {
    return __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay)),
                     __dmul_rn(__dsub_rn(by, ay), __dsub_rn(px, ax)));
}

struct Tri2 {
    double x[3], y[3];
};

__device__ __forceinline__ Tri2 load_tri(const double* xy, int64_t nv, const int32_t* tri,
                                         int64_t nt, int64_t k) {
    Tri2 t;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int32_t v = tri[c * nt + k];
        t.x[c] = xy[v];
        t.y[c] = xy[nv + v];
    }
    return t;
}

// barycentric coordinates of (px, py) in t (det = orient of t's vertices, non-zero)
__device__ __forceinline__ void bary(const Tri2& t, double det, double px, double py, double* l) {
    l[1] = __ddiv_rn(orient2(t.x[0], t.y[0], px, py, t.x[2], t.y[2]), det);
    l[2] = __ddiv_rn(orient2(t.x[0], t.y[0], t.x[1], t.y[1], px, py), det);
    l[0] = __dsub_rn(__dsub_rn(1.0, l[1]), l[2]);
}

struct ProjArgs {
    // source mesh (with its grid of triangles per cell)
    Grid g;
    int64_t snv, snt;
    const double* sxy;
    const int32_t* stri;
    const int8_t* ssign;
    const int32_t* cell_start;
    const int32_t* items;
    const double* fs;   // source nodal field
    // target mesh
    int64_t tnv, tnt;
    const double* txy;
    const int32_t* ttri;
    const int8_t* tsign;
    double* tri_b;      // [tnt][3] contributions to b at T's vertices
    double* tri_area;   // [tnt] area of the supermesh pieces in T
    unsigned long long* pairs;
};

__global__ void __launch_bounds__(PJ_THREADS) k_supermesh_rhs(ProjArgs A) {
    const Grid& g = A.g;
    unsigned long long npairs = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A.tnt;
         k += (int64_t)gridDim.x * blockDim.x) {
        double bl[3] = {0.0, 0.0, 0.0}, area = 0.0;
        const int sgn = A.tsign[k];
        if (sgn != 0) {
            Tri2 T = load_tri(A.txy, A.tnv, A.ttri, A.tnt, k);
            int perm[3] = {0, 1, 2};   // T counter-clockwise
            if (sgn < 0) {
                perm[1] = 2;
                perm[2] = 1;
            }
            Tri2 Tc;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                Tc.x[c] = T.x[perm[c]];
                Tc.y[c] = T.y[perm[c]];
            }
            const double tdet = orient2(Tc.x[0], Tc.y[0], Tc.x[1], Tc.y[1], Tc.x[2], Tc.y[2]);
            const double tx0 = fmin(Tc.x[0], fmin(Tc.x[1], Tc.x[2]));
            const double tx1 = fmax(Tc.x[0], fmax(Tc.x[1], Tc.x[2]));
            const double ty0 = fmin(Tc.y[0], fmin(Tc.y[1], Tc.y[2]));
            const double ty1 = fmax(Tc.y[0], fmax(Tc.y[1], Tc.y[2]));
            const int cx0 = grid_cell(tx0, g.lo[0], g.inv_h, g.n[0]);
            const int cx1 = grid_cell(tx1, g.lo[0], g.inv_h, g.n[0]);
            const int cy0 = grid_cell(ty0, g.lo[1], g.inv_h, g.n[1]);
            const int cy1 = grid_cell(ty1, g.lo[1], g.inv_h, g.n[1]);
            for (int cy = cy0; cy <= cy1; cy++)
                for (int cx = cx0; cx <= cx1; cx++) {
                    const int64_t c = (int64_t)cy * g.n[0] + cx;
                    for (int it = A.cell_start[c]; it < A.cell_start[c + 1]; it++) {
                        const int32_t si = A.items[it];
                        if (A.ssign[si] == 0) continue;
                        const Tri2 S = load_tri(A.sxy, A.snv, A.stri, A.snt, si);
                        const double sx0 = fmin(S.x[0], fmin(S.x[1], S.x[2]));
                        const double sx1 = fmax(S.x[0], fmax(S.x[1], S.x[2]));
                        const double sy0 = fmin(S.y[0], fmin(S.y[1], S.y[2]));
                        const double sy1 = fmax(S.y[0], fmax(S.y[1], S.y[2]));
                        if (sx0 > tx1 || sx1 < tx0 || sy0 > ty1 || sy1 < ty0) continue;
                        // the pair is handled in the cell of the boxes' lower-left corner only
                        if (grid_cell(fmax(sx0, tx0), g.lo[0], g.inv_h, g.n[0]) != cx ||
                            grid_cell(fmax(sy0, ty0), g.lo[1], g.inv_h, g.n[1]) != cy)
                            continue;
                        // clip S by the half-planes left of T's edges
                        double px[8], py[8], qx[8], qy[8];
                        int n = 3;
#pragma unroll
                        for (int c3 = 0; c3 < 3; c3++) {
                            px[c3] = S.x[c3];
                            py[c3] = S.y[c3];
                        }
#pragma unroll
                        for (int e = 0; e < 3; e++) {
                            const double ax = Tc.x[e], ay = Tc.y[e];
                            const double bx = Tc.x[(e + 1) % 3], by = Tc.y[(e + 1) % 3];
                            int m = 0;
                            for (int i = 0; i < n; i++) {
                                const int i1 = i + 1 < n ? i + 1 : 0;
                                const double sp = orient2(ax, ay, bx, by, px[i], py[i]);
                                const double sq = orient2(ax, ay, bx, by, px[i1], py[i1]);
                                if (sp >= 0.0 && m < 8) {
                                    qx[m] = px[i];
                                    qy[m] = py[i];
                                    m++;
                                }
                                if ((sp >= 0.0) != (sq >= 0.0) && m < 8) {
                                    const double t = __ddiv_rn(sp, __dsub_rn(sp, sq));
                                    qx[m] = __dadd_rn(px[i], __dmul_rn(t, __dsub_rn(px[i1], px[i])));
                                    qy[m] = __dadd_rn(py[i], __dmul_rn(t, __dsub_rn(py[i1], py[i])));
                                    m++;
                                }
                            }
                            n = m;
                            for (int i = 0; i < n; i++) {
                                px[i] = qx[i];
                                py[i] = qy[i];
                            }
                            if (n < 3) break;
                        }
                        if (n < 3) continue;
                        ++npairs;
                        const double sdet = orient2(S.x[0], S.y[0], S.x[1], S.y[1], S.x[2], S.y[2]);
                        const double f0 = A.fs[A.stri[si]], f1 = A.fs[A.stri[A.snt + si]],
                                     f2 = A.fs[A.stri[2 * A.snt + si]];
                        for (int i = 1; i + 1 < n; i++) {
                            const double ar =
                                0.5 * fabs(orient2(px[0], py[0], px[i], py[i], px[i + 1], py[i + 1]));
                            if (ar == 0.0) continue;
                            area += ar;
                            const int vi[3] = {0, i, i + 1};
#pragma unroll
                            for (int e = 0; e < 3; e++) {
                                const int a0 = vi[e], a1 = vi[(e + 1) % 3];
                                const double mx = 0.5 * __dadd_rn(px[a0], px[a1]);
                                const double my = 0.5 * __dadd_rn(py[a0], py[a1]);
                                double ls[3], lt[3];
                                bary(S, sdet, mx, my, ls);
                                bary(Tc, tdet, mx, my, lt);
                                const double fv = ls[0] * f0 + ls[1] * f1 + ls[2] * f2;
                                const double wq = (ar / 3.0) * fv;
#pragma unroll
                                for (int c3 = 0; c3 < 3; c3++) bl[perm[c3]] += wq * lt[c3];
                            }
                        }
                    }
                }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) A.tri_b[3 * k + c] = bl[c];
        A.tri_area[k] = area;
    }
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if ((threadIdx.x & 31) == 0 && npairs) atomicAdd(A.pairs, npairs);
}

// vertex -> (triangle, corner) lists of a mesh, ascending by triangle within a vertex
__global__ void k_adj_count(int64_t nt, const int32_t* __restrict__ tri, int32_t* __restrict__ cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; c++) atomicAdd(&cnt[tri[c * nt + k]], 1);
}
__global__ void k_adj_fill(int64_t nt, const int32_t* __restrict__ tri,
                           const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                           int32_t* __restrict__ items) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int32_t v = tri[c * nt + k];
            items[start[v] + atomicAdd(&fill[v], 1)] = (int32_t)(3 * k + c);
        }
}
__global__ void k_adj_sort(int64_t nv, const int32_t* __restrict__ start, int32_t* items) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int a = start[v], b = start[v + 1];
        for (int i = a + 1; i < b; i++) {
            const int32_t x = items[i];
            int j = i - 1;
            while (j >= a && items[j] > x) {
                items[j + 1] = items[j];
                j--;
            }
            items[j + 1] = x;
        }
    }
}

// per-triangle |T| / 12
__global__ void k_tri_w(int64_t nv, const double* __restrict__ xy, int64_t nt,
                        const int32_t* __restrict__ tri, double* __restrict__ w) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const Tri2 t = load_tri(xy, nv, tri, nt, k);
        w[k] = fabs(orient2(t.x[0], t.y[0], t.x[1], t.y[1], t.x[2], t.y[2])) / 24.0;
    }
}

// b_A = sum over A's triangles of their corner contribution; diag_A = sum of |T|/6
__global__ void k_vertex_gather(int64_t nv, const int32_t* __restrict__ start,
                                const int32_t* __restrict__ items, const double* __restrict__ tri_b,
                                const double* __restrict__ w, double* __restrict__ b,
                                double* __restrict__ diag) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0, d = 0.0;
        for (int i = start[v]; i < start[v + 1]; i++) {
            const int32_t e = items[i];
            s += tri_b[e];
            d += 2.0 * w[e / 3];
        }
        b[v] = s;
        diag[v] = d;
    }
}

// q = M p and the block's partial sum of p . q
__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = PJ_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(PJ_THREADS) k_mass_apply(
    int64_t nv, int64_t nt, const int32_t* __restrict__ tri, const double* __restrict__ w,
    const int32_t* __restrict__ start, const int32_t* __restrict__ items,
    const double* __restrict__ p, double* __restrict__ q, double* __restrict__ part) {
    __shared__ double sh[PJ_THREADS];
    double acc = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double pv = p[v];
        double s = 0.0;
        for (int i = start[v]; i < start[v + 1]; i++) {
            const int64_t k = items[i] / 3;
            s += w[k] * (pv + p[tri[k]] + p[tri[nt + k]] + p[tri[2 * nt + k]]);
        }
        q[v] = s;
        acc += pv * s;
    }
    const double r = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// CG scalars on the device: s[0] = r.z, s[1] = alpha, s[2] = beta, s[3] = r.r, s[4] = b.b
__global__ void __launch_bounds__(PJ_THREADS) k_cg_alpha(const double* __restrict__ part, int n,
                                                         double* s) {
    __shared__ double sh[PJ_THREADS];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
    const double pq = block_sum(a, sh);
    if (threadIdx.x == 0) s[1] = pq != 0.0 ? s[0] / pq : 0.0;
}

// x += alpha p, r -= alpha q, z = r / diag; partial sums of r.z and r.r
__global__ void __launch_bounds__(PJ_THREADS) k_cg_update(
    int64_t nv, const double* __restrict__ s, const double* __restrict__ p,
    const double* __restrict__ q, const double* __restrict__ diag, double* __restrict__ x,
    double* __restrict__ r, double* __restrict__ z, double* __restrict__ part) {
    __shared__ double sh[PJ_THREADS];
    const double alpha = s[1];
    double rz = 0.0, rr = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        x[v] += alpha * p[v];
        const double rv = r[v] - alpha * q[v];
        r[v] = rv;
        const double zv = rv / diag[v];
        z[v] = zv;
        rz += rv * zv;
        rr += rv * rv;
    }
    const double a = block_sum(rz, sh);
    const double b = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[PJ_BLOCKS + blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(PJ_THREADS) k_cg_beta(const double* __restrict__ part, int n,
                                                        double* s) {
    __shared__ double sh[PJ_THREADS];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += part[i];
        b += part[PJ_BLOCKS + i];
    }
    const double rz = block_sum(a, sh);
    const double rr = block_sum(b, sh);
    if (threadIdx.x == 0) {
        s[2] = s[0] != 0.0 ? rz / s[0] : 0.0;
        s[0] = rz;
        s[3] = rr;
    }
}

// p = z + beta p
__global__ void k_cg_direction(int64_t nv, const double* __restrict__ s,
                               const double* __restrict__ z, double* __restrict__ p) {
    const double beta = s[2];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        p[v] = z[v] + beta * p[v];
}

// start: x = b / (row sums of M) (the lumped solution), r = b - M x, z = r / diag, p = z;
// partial sums of r.z, r.r and b.b
__global__ void __launch_bounds__(PJ_THREADS) k_cg_start(
    int64_t nv, const double* __restrict__ b, const double* __restrict__ mx,
    const double* __restrict__ diag, double* __restrict__ r, double* __restrict__ z,
    double* __restrict__ p, double* __restrict__ part) {
    __shared__ double sh[PJ_THREADS];
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double rv = b[v] - mx[v];
        r[v] = rv;
        const double zv = rv / diag[v];
        z[v] = zv;
        p[v] = zv;
        rz += rv * zv;
        rr += rv * rv;
        bb += b[v] * b[v];
    }
    const double a = block_sum(rz, sh);
    const double c = block_sum(rr, sh);
    const double d = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[PJ_BLOCKS + blockIdx.x] = c;
        part[2 * PJ_BLOCKS + blockIdx.x] = d;
    }
}

__global__ void __launch_bounds__(PJ_THREADS) k_cg_start_sums(const double* __restrict__ part,
                                                              int n, double* s) {
    __shared__ double sh[PJ_THREADS];
    double a = 0.0, c = 0.0, d = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += part[i];
        c += part[PJ_BLOCKS + i];
        d += part[2 * PJ_BLOCKS + i];
    }
    const double rz = block_sum(a, sh);
    const double rr = block_sum(c, sh);
    const double bb = block_sum(d, sh);
    if (threadIdx.x == 0) {
        s[0] = rz;
        s[3] = rr;
        s[4] = bb;
    }
}

// lumped start: x = b / sum_B M_AB, with sum_B M_AB = sum over A's triangles of |T| / 3
__global__ void k_lumped(int64_t nv, const int32_t* __restrict__ start,
                         const int32_t* __restrict__ items, const double* __restrict__ w,
                         const double* __restrict__ b, double* __restrict__ x) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int i = start[v]; i < start[v + 1]; i++) m += 4.0 * w[items[i] / 3];
        x[v] = m > 0.0 ? b[v] / m : 0.0;
    }
}

__global__ void k_sum_fixed(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
    __shared__ double sh[PJ_THREADS];
    double a = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a += v[i];
    const double r = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

}  // namespace

void mesh_adjacency(MeshImpl& M, cudaStream_t s) {
    if (M.adj_start.p) return;
    const int64_t nv = M.nv, nt = M.ntri;
    DBuf cnt(sizeof(int32_t) * (nv + 1), s);
    PCMS_CU(cudaMemsetAsync(cnt.p, 0, cnt.bytes, s));
    M.adj_start.alloc(sizeof(int32_t) * (nv + 1), s);
    M.adj.alloc(sizeof(int32_t) * std::max<int64_t>(3 * nt, 1), s);
    M.tri_w.alloc(sizeof(double) * std::max<int64_t>(nt, 1), s);
    if (nt > 0) {
        PCMS_TRACE("mesh_adjacency_count", s);
        k_adj_count<<<pj_blocks(nt), PJ_THREADS, 0, s>>>(nt, M.tri.as<int32_t>(), cnt.as<int32_t>());
    }
    exclusive_scan<int32_t>(cnt.as<int32_t>(), M.adj_start.as<int32_t>(), nv, s);
    PCMS_CU(cudaMemsetAsync(cnt.p, 0, cnt.bytes, s));
    if (nt > 0) {
        {
            PCMS_TRACE("mesh_adjacency_fill", s);
            k_adj_fill<<<pj_blocks(nt), PJ_THREADS, 0, s>>>(nt, M.tri.as<int32_t>(),
                                                            M.adj_start.as<int32_t>(),
                                                            cnt.as<int32_t>(), M.adj.as<int32_t>());
        }
        {
            PCMS_TRACE("mesh_adjacency_sort", s);
            k_adj_sort<<<pj_blocks(nv), PJ_THREADS, 0, s>>>(nv, M.adj_start.as<int32_t>(),
                                                            M.adj.as<int32_t>());
        }
        {
            PCMS_TRACE("mesh_triangle_weights", s);
            k_tri_w<<<pj_blocks(nt), PJ_THREADS, 0, s>>>(nv, M.xy.as<double>(), nt,
                                                         M.tri.as<int32_t>(), M.tri_w.as<double>());
        }
    }
    PCMS_LAUNCH_CHECK("mesh_adjacency");
}

ProjectionResult l2_project(const MeshImpl& S, const double* fs, MeshImpl& T, double* ft,
                            double tol, int max_iter, cudaStream_t s) {
    ProjectionResult res{};
    const int64_t nv = T.nv, nt = T.ntri;
    mesh_adjacency(T, s);
    DBuf trib(sizeof(double) * 3 * std::max<int64_t>(nt, 1), s);
    DBuf tarea(sizeof(double) * std::max<int64_t>(nt, 1), s);
    DBuf ctl(sizeof(unsigned long long) + sizeof(double) * 8, s);
    auto* pairs = ctl.as<unsigned long long>();
    double* sc = (double*)(pairs + 1);
    PCMS_CU(cudaMemsetAsync(ctl.p, 0, ctl.bytes, s));
    const int64_t nn = std::max<int64_t>(nv, 1);
    DBuf vec(sizeof(double) * 6 * nn, s);
    double* b = vec.as<double>();
    double* diag = b + nn;
    double* r = diag + nn;
    double* z = r + nn;
    double* p = z + nn;
    double* q = p + nn;
    DBuf part(sizeof(double) * 3 * PJ_BLOCKS, s);
    if (nt > 0) {
        ProjArgs A{};
        A.g = S.g;
        A.snv = S.nv;
        A.snt = S.ntri;
        A.sxy = S.xy.as<double>();
        A.stri = S.tri.as<int32_t>();
        A.ssign = S.tsign.as<int8_t>();
        A.cell_start = S.cell_start.as<int32_t>();
        A.items = S.items.as<int32_t>();
        A.fs = fs;
        A.tnv = T.nv;
        A.tnt = T.ntri;
        A.txy = T.xy.as<double>();
        A.ttri = T.tri.as<int32_t>();
        A.tsign = T.tsign.as<int8_t>();
        A.tri_b = trib.as<double>();
        A.tri_area = tarea.as<double>();
        A.pairs = pairs;
        PCMS_TRACE("projection_supermesh_rhs", s);
        k_supermesh_rhs<<<pj_blocks(nt), PJ_THREADS, 0, s>>>(A);
    }
    PCMS_LAUNCH_CHECK("k_supermesh_rhs");
    if (nv == 0) return res;
    {
        PCMS_TRACE("projection_gather", s);
        k_vertex_gather<<<pj_blocks(nv), PJ_THREADS, 0, s>>>(nv, T.adj_start.as<int32_t>(),
                                                             T.adj.as<int32_t>(), trib.as<double>(),
                                                             T.tri_w.as<double>(), b, diag);
    }
    // supermesh area: fixed-order sum
    {
        PCMS_TRACE("projection_area_sum", s);
        k_sum_fixed<<<PJ_BLOCKS, PJ_THREADS, 0, s>>>(tarea.as<double>(), nt, part.as<double>());
    }
    {
        PCMS_TRACE("projection_area_sum", s);
        k_sum_fixed<<<1, PJ_THREADS, 0, s>>>(part.as<double>(), PJ_BLOCKS, sc + 6);
    }
    const int nb = PJ_BLOCKS;
    const int32_t* as = T.adj_start.as<int32_t>();
    const int32_t* ai = T.adj.as<int32_t>();
    const double* w = T.tri_w.as<double>();
    const int32_t* tri = T.tri.as<int32_t>();
    {
        PCMS_TRACE("projection_cg_lumped", s);
        k_lumped<<<pj_blocks(nv), PJ_THREADS, 0, s>>>(nv, as, ai, w, b, ft);
    }
    {
        PCMS_TRACE("projection_mass_apply", s);
        k_mass_apply<<<nb, PJ_THREADS, 0, s>>>(nv, nt, tri, w, as, ai, ft, q, part.as<double>());
    }
    {
        PCMS_TRACE("projection_cg_start", s);
        k_cg_start<<<nb, PJ_THREADS, 0, s>>>(nv, b, q, diag, r, z, p, part.as<double>());
    }
    {
        PCMS_TRACE("projection_cg_scalars", s);
        k_cg_start_sums<<<1, PJ_THREADS, 0, s>>>(part.as<double>(), nb, sc);
    }
    PCMS_LAUNCH_CHECK("projection_cg_start");
    double h[8];
    PCMS_CU(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaMemcpyAsync(&res.pairs, pairs, sizeof(res.pairs), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    res.supermesh_area = h[6];
    const double bb = h[4];
    double rr = h[3];
    int it = 0;
    const double stop = tol * tol * bb;
    while (it < max_iter && rr > stop && bb > 0.0) {
        for (int k = 0; k < CG_CHECK && it < max_iter; k++, it++) {
            {
                PCMS_TRACE("projection_mass_apply", s);
                k_mass_apply<<<nb, PJ_THREADS, 0, s>>>(nv, nt, tri, w, as, ai, p, q, part.as<double>());
            }
            {
                PCMS_TRACE("projection_cg_scalars", s);
                k_cg_alpha<<<1, PJ_THREADS, 0, s>>>(part.as<double>(), nb, sc);
            }
            {
                PCMS_TRACE("projection_cg_update", s);
                k_cg_update<<<nb, PJ_THREADS, 0, s>>>(nv, sc, p, q, diag, ft, r, z, part.as<double>());
            }
            {
                PCMS_TRACE("projection_cg_scalars", s);
                k_cg_beta<<<1, PJ_THREADS, 0, s>>>(part.as<double>(), nb, sc);
            }
            {
                PCMS_TRACE("projection_cg_direction", s);
                k_cg_direction<<<pj_blocks(nv), PJ_THREADS, 0, s>>>(nv, sc, z, p);
            }
        }
        PCMS_LAUNCH_CHECK("projection_cg");
        PCMS_CU(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
        rr = h[3];
    }
    res.iterations = it;
    res.rel_residual = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    return res;
}

}  // namespace pcms
