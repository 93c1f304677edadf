// mesh.cu -- point localization in a triangle mesh with lowest-order topological
// classification, and barycentric (parametric) interpolation (Sec. 3.3).
//
// Search structure (Sec. 3.3, single-level uniform grid): every triangle is listed in each
// cell its bounding box overlaps; lists are sorted by triangle id. Cell coordinates of
// bounding-box corners and of query points use the same monotone expression
// floor((x - lo) * inv_h), so a triangle whose closure contains p is always listed in p's
// cell. Scanning the list in ascending id and stopping at the first triangle whose closure
// contains p yields the smallest such id, which makes the answer independent of traversal
// order (the consistency requirement of Sec. 3.3).
//
// Orientation signs are exact: a floating-point filter with Shewchuk's error bound
// (3 + 16 eps) eps (|detleft| + |detright|) decides almost every case; the rest is
// evaluated exactly by splitting each coordinate difference and each product into
// non-overlapping double expansions (two-diff, FMA-based two-product, two-sum) and taking
// the sign of the largest component of their exact sum.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pcms_internal.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

int blocks_for(int64_t n, int threads, int per_sm = 32) {
    int64_t need = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * per_sm));
}

__device__ __forceinline__ int mesh_cell(double x, double lo, double inv_h, int n) {
    double f = floor((x - lo) * inv_h);
    f = fmin(fmax(f, 0.0), (double)(n - 1));
    return (int)f;
}

// ---------------------------------------------------------------------- exact orientation
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}
__device__ __forceinline__ void two_diff(double a, double b, double& s, double& e) {
    s = __dsub_rn(a, b);
    double bv = __dsub_rn(a, s);
    double av = __dadd_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(bv, b));
}
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
    p = __dmul_rn(a, b);
    e = fma(a, b, -p);
}

// exact sign of (ax-cx)(by-cy) - (ay-cy)(bx-cx)
__device__ __noinline__ int orient_exact(double ax, double ay, double bx, double by, double cx,
                                         double cy) {
    double u[2], v[2], w[2], z[2];   // ax-cx, by-cy, ay-cy, bx-cx as hi+lo
    two_diff(ax, cx, u[0], u[1]);
    two_diff(by, cy, v[0], v[1]);
    two_diff(ay, cy, w[0], w[1]);
    two_diff(bx, cx, z[0], z[1]);
    double e[17];
    int n = 0;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int neg = 0; neg < 2; neg++) {
                double p, q;
                if (neg == 0) two_prod(u[i], v[j], p, q);
                else two_prod(-w[i], z[j], p, q);
                double terms[2] = {q, p};
                for (int t = 0; t < 2; t++) {
                    double acc = terms[t];
                    for (int k = 0; k < n; k++) {
                        double s, h;
                        two_sum(acc, e[k], s, h);
                        e[k] = h;
                        acc = s;
                    }
                    e[n++] = acc;
                }
            }
    for (int k = n - 1; k >= 0; k--) {
        if (e[k] > 0.0) return 1;
        if (e[k] < 0.0) return -1;
    }
    return 0;
}

__device__ __forceinline__ int orient_sign(double ax, double ay, double bx, double by, double cx,
                                           double cy) {
    const double detleft = __dmul_rn(__dsub_rn(ax, cx), __dsub_rn(by, cy));
    const double detright = __dmul_rn(__dsub_rn(ay, cy), __dsub_rn(bx, cx));
    const double det = __dsub_rn(detleft, detright);
    double detsum;
    if (detleft > 0.0) {
        if (detright <= 0.0) return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
        detsum = detleft + detright;
    } else if (detleft < 0.0) {
        if (detright >= 0.0) return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
        detsum = -detleft - detright;
    } else {
        return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
    }
    const double errbound = 3.3306690738754716e-16 * detsum;   // (3 + 16 eps) eps, eps = 2^-53
    if (det >= errbound) return 1;
    if (-det >= errbound) return -1;
    return orient_exact(ax, ay, bx, by, cx, cy);
}

// FP32 filter for orient_sign(a, b, p): +1 or -1 when the sign is certain, 0 when it is not.
// Points are FP32 hi/lo pairs relative to a common origin (a = (A.x, A.y) + (A.z, A.w)), so
// each difference a - p, formed as (a_hi - p_hi) + (a_lo - p_lo), is within 2u|d| + delta of
// the exact one (u = 2^-24; delta = 2^-44 x the extent covers the split of the FP64 inputs
// and the lo parts' rounding). Propagating that through the two products and the
// subtraction gives |det - det_exact| <= 6.01u (|l| + |r|) + 1.01 delta (|X|+|Y|+|Z|+|W|)
// + 2 delta^2; the bound below has at least 25% to spare on every term, and 1e-37 covers
// underflow. Points on an edge (det_exact = 0) always fail the test and are decided by the
// FP64 filter and the exact expansion.
__device__ __forceinline__ int orient_filter32(float4 A, float4 B, float phx, float phy,
                                               float plx, float ply, float delta) {
    const float X = __fadd_rn(__fsub_rn(A.x, phx), __fsub_rn(A.z, plx));   // ax - px
    const float Z = __fadd_rn(__fsub_rn(A.y, phy), __fsub_rn(A.w, ply));   // ay - py
    const float W = __fadd_rn(__fsub_rn(B.x, phx), __fsub_rn(B.z, plx));   // bx - px
    const float Y = __fadd_rn(__fsub_rn(B.y, phy), __fsub_rn(B.w, ply));   // by - py
    const float l = __fmul_rn(X, Y), r = __fmul_rn(Z, W);
    const float det = __fsub_rn(l, r);
    const float bound = 4.76837158e-07f * (fabsf(l) + fabsf(r)) +
                        2.0f * delta * (fabsf(X) + fabsf(Y) + fabsf(Z) + fabsf(W)) +
                        3.0f * delta * delta + 1e-37f;
    if (det > bound) return 1;
    if (det < -bound) return -1;
    return 0;
}

__global__ void k_vertex_hilo(int64_t nv, const double* __restrict__ xy, double ox, double oy,
                              float4* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double rx = xy[i] - ox, ry = xy[nv + i] - oy;
        const float hx = (float)rx, hy = (float)ry;
        out[i] = make_float4(hx, hy, (float)(rx - (double)hx), (float)(ry - (double)hy));
    }
}

__device__ __forceinline__ double orient_fp(double ax, double ay, double bx, double by, double cx,
                                            double cy) {
    return __dsub_rn(__dmul_rn(__dsub_rn(ax, cx), __dsub_rn(by, cy)),
                     __dmul_rn(__dsub_rn(ay, cy), __dsub_rn(bx, cx)));
}

// ---------------------------------------------------------------------- build kernels
// Cell ranges in FP32 (use32): cell coordinates (hi + lo) * (1/h) of the vertices' hi/lo
// pairs (relative to the grid origin), within about 2^-22 n < 0.005 cells of the exact ones
// (n <= 16384 cells per axis); each range is widened by CELL_MARGIN, above twice that, so it
// covers every cell that the FP64 cell of a point inside the triangle, or its FP32 cell in
// k_locate, can be. Wider ranges only add candidates.
constexpr float CELL_MARGIN = 1.f / 64.f;

__device__ __forceinline__ int cell32(float c, int n) {
    return min(max(__float2int_rd(c), 0), n - 1);
}

__global__ void k_tri_prep(int64_t nv, const double* __restrict__ xy, int64_t nt,
                           const int32_t* __restrict__ tri, Grid g, int32_t* __restrict__ count,
                           int8_t* __restrict__ tsign, int4* __restrict__ trect,
                           unsigned long long* bad_ids, const float4* __restrict__ vhl,
                           int use32, float delta, float ihf) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t i0 = tri[k], i1 = tri[nt + k], i2 = tri[2 * nt + k];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
            atomicAdd(bad_ids, 1ull);
            tsign[k] = 0;
            trect[k] = make_int4(1, 1, 0, 0);   // empty
            continue;
        }
        int s = 0, cx0, cx1, cy0, cy1;
        if (use32) {
            // orientation: the FP32 filter of orient(v0, v1, v2), FP64 and exact when undecided
            const float4 A = vhl[i0], B = vhl[i1], C = vhl[i2];
            s = orient_filter32(A, B, C.x, C.y, C.z, C.w, delta);
            if (s == 0)
                s = orient_sign(xy[i0], xy[nv + i0], xy[i1], xy[nv + i1], xy[i2], xy[nv + i2]);
            const float ax = (A.x + A.z) * ihf, bx = (B.x + B.z) * ihf, cx = (C.x + C.z) * ihf;
            const float ay = (A.y + A.w) * ihf, by = (B.y + B.w) * ihf, cy = (C.y + C.w) * ihf;
            cx0 = cell32(fminf(ax, fminf(bx, cx)) - CELL_MARGIN, g.n[0]);
            cx1 = cell32(fmaxf(ax, fmaxf(bx, cx)) + CELL_MARGIN, g.n[0]);
            cy0 = cell32(fminf(ay, fminf(by, cy)) - CELL_MARGIN, g.n[1]);
            cy1 = cell32(fmaxf(ay, fmaxf(by, cy)) + CELL_MARGIN, g.n[1]);
        } else {
            double x0 = xy[i0], y0 = xy[nv + i0], x1 = xy[i1], y1 = xy[nv + i1];
            double x2 = xy[i2], y2 = xy[nv + i2];
            s = orient_sign(x0, y0, x1, y1, x2, y2);
            cx0 = mesh_cell(fmin(x0, fmin(x1, x2)), g.lo[0], g.inv_h, g.n[0]);
            cx1 = mesh_cell(fmax(x0, fmax(x1, x2)), g.lo[0], g.inv_h, g.n[0]);
            cy0 = mesh_cell(fmin(y0, fmin(y1, y2)), g.lo[1], g.inv_h, g.n[1]);
            cy1 = mesh_cell(fmax(y0, fmax(y1, y2)), g.lo[1], g.inv_h, g.n[1]);
        }
        tsign[k] = (int8_t)s;
        if (s == 0) {
            trect[k] = make_int4(1, 1, 0, 0);
            continue;
        }
        trect[k] = make_int4(cx0, cy0, cx1, cy1);
        for (int cy = cy0; cy <= cy1; cy++)
            for (int cx = cx0; cx <= cx1; cx++) atomicAdd(&count[(int64_t)cy * g.n[0] + cx], 1);
    }
}

__global__ void k_tri_fill(int64_t nt, Grid g, const int4* __restrict__ trect,
                           const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                           int32_t* __restrict__ items) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        int4 r = trect[k];
        for (int cy = r.y; cy <= r.w; cy++)
            for (int cx = r.x; cx <= r.z; cx++) {
                int64_t c = (int64_t)cy * g.n[0] + cx;
                int pos = start[c] + atomicAdd(&fill[c], 1);
                items[pos] = (int32_t)k;
            }
    }
}

// odd-even transposition sort of N registers (N rounds of compare-exchanges)
template <int N>
__device__ __forceinline__ void sort_regs(int32_t (&v)[N]) {
#pragma unroll
    for (int r = 0; r < N; r++) {
#pragma unroll
        for (int j = r & 1; j + 1 < N; j += 2) {
            const int32_t lo = min(v[j], v[j + 1]), hi = max(v[j], v[j + 1]);
            v[j] = lo;
            v[j + 1] = hi;
        }
    }
}

// the cell's n <= N items loaded together, sorted in registers (padding sorts last), stored
template <int N>
__device__ __forceinline__ void sort_cell_regs(int32_t* items, int a, int n) {
    int32_t v[N];
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = i < n ? items[a + i] : INT32_MAX;
    sort_regs<N>(v);
#pragma unroll
    for (int i = 0; i < N; i++)
        if (i < n) items[a + i] = v[i];
}

// Each cell's triangle IDs ascending (the fill order is that of atomics): one thread per cell;
// up to 16 items are sorted in registers, longer cells by insertion in place.
__global__ void k_cell_sort(int64_t ncell, const int32_t* __restrict__ start, int32_t* items) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int a = start[c], b = start[c + 1], n = b - a;
        if (n <= 1) continue;
        if (n <= 8) {
            sort_cell_regs<8>(items, a, n);
            continue;
        }
        if (n <= 16) {
            sort_cell_regs<16>(items, a, n);
            continue;
        }
        for (int i = a + 1; i < b; i++) {
            int32_t v = items[i];
            int j = i - 1;
            while (j >= a && items[j] > v) {
                items[j + 1] = items[j];
                j--;
            }
            items[j + 1] = v;
        }
    }
}

// ---------------------------------------------------------------------- query kernel
__global__ void __launch_bounds__(256) k_locate(Grid g, double bx0, double by0, double bx1,
                                                double by1, int64_t nv,
                                                const double* __restrict__ xy, int64_t ntri,
                                                const int32_t* __restrict__ tri,
                                                const int8_t* __restrict__ tsign,
                                                const int32_t* __restrict__ start,
                                                const int32_t* __restrict__ items,
                                                const float4* __restrict__ vhl, double ox,
                                                double oy, float delta, int use32, float ihf,
                                                const double* __restrict__ pts, int64_t n,
                                                const double* __restrict__ field,
                                                int32_t* __restrict__ elem,
                                                int8_t* __restrict__ edim,
                                                double* __restrict__ vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double px = pts[i], py = pts[n + i];
        int32_t found = -1;
        int nz = 0;
        int32_t v0 = 0, v1 = 0, v2 = 0;
        if (px >= bx0 && px <= bx1 && py >= by0 && py <= by1) {
            // the point in the FP32 filter's frame (the origin is the grid's)
            const double rx = px - ox, ry = py - oy;
            const float phx = (float)rx, phy = (float)ry;
            const float plx = (float)(rx - (double)phx), ply = (float)(ry - (double)phy);
            // its cell: in FP32 when the triangles' ranges were (widened by CELL_MARGIN)
            const int64_t c =
                use32 ? (int64_t)cell32((phy + ply) * ihf, g.n[1]) * g.n[0] +
                            cell32((phx + plx) * ihf, g.n[0])
                      : (int64_t)mesh_cell(py, g.lo[1], g.inv_h, g.n[1]) * g.n[0] +
                            mesh_cell(px, g.lo[0], g.inv_h, g.n[0]);
            const int a = start[c], b = start[c + 1];
            for (int it = a; it < b; it++) {
                const int32_t k = items[it];
                const int s = tsign[k];
                const int32_t i0 = tri[k], i1 = tri[ntri + k], i2 = tri[2 * ntri + k];
                int o0 = 0, o1 = 0, o2 = 0;
                if (use32) {
                    const float4 A = vhl[i0], B = vhl[i1], C = vhl[i2];
                    o0 = orient_filter32(B, C, phx, phy, plx, ply, delta);
                    if (o0 * s < 0) continue;
                    o1 = orient_filter32(C, A, phx, phy, plx, ply, delta);
                    if (o1 * s < 0) continue;
                    o2 = orient_filter32(A, B, phx, phy, plx, ply, delta);
                    if (o2 * s < 0) continue;
                }
                if (o0 == 0 || o1 == 0 || o2 == 0) {   // undecided in FP32: FP64 filter, then exact
                    const double x0 = xy[i0], y0 = xy[nv + i0];
                    const double x1 = xy[i1], y1 = xy[nv + i1];
                    const double x2 = xy[i2], y2 = xy[nv + i2];
                    if (o0 == 0) o0 = orient_sign(x1, y1, x2, y2, px, py);
                    if (o0 * s < 0) continue;
                    if (o1 == 0) o1 = orient_sign(x2, y2, x0, y0, px, py);
                    if (o1 * s < 0) continue;
                    if (o2 == 0) o2 = orient_sign(x0, y0, x1, y1, px, py);
                    if (o2 * s < 0) continue;
                }
                found = k;
                nz = (o0 == 0) + (o1 == 0) + (o2 == 0);
                v0 = i0; v1 = i1; v2 = i2;
                break;
            }
        }
        elem[i] = found;
        if (edim) edim[i] = (int8_t)(found < 0 ? -1 : 2 - nz);
        if (vals) {
            double v = __longlong_as_double(0x7ff8000000000000LL);
            if (found >= 0) {
                const double x0 = xy[v0], y0 = xy[nv + v0];
                const double x1 = xy[v1], y1 = xy[nv + v1];
                const double x2 = xy[v2], y2 = xy[nv + v2];
                // one reciprocal of the doubled area for both coordinates (within 2 ulp of the
                // quotients; the FP64 pipe is this kernel's bound)
                const double rarea = recip64(orient_fp(x0, y0, x1, y1, x2, y2));
                const double l0 = __dmul_rn(orient_fp(px, py, x1, y1, x2, y2), rarea);
                const double l1 = __dmul_rn(orient_fp(x0, y0, px, py, x2, y2), rarea);
                const double l2 = __dsub_rn(__dsub_rn(1.0, l0), l1);
                v = __dadd_rn(__dadd_rn(__dmul_rn(l0, field[v0]), __dmul_rn(l1, field[v1])),
                              __dmul_rn(l2, field[v2]));
            }
            vals[i] = v;
        }
    }
}

}  // namespace

void mesh_create(MeshImpl& M, const double* xy, int64_t nv, const int32_t* tri, int64_t ntri) {
    cudaStream_t s = M.stream;
    M.nv = nv;
    M.ntri = ntri;
    M.xy.alloc(sizeof(double) * 2 * std::max<int64_t>(nv, 1), s);
    M.tri.alloc(sizeof(int32_t) * 3 * std::max<int64_t>(ntri, 1), s);
    if (nv > 0) PCMS_CU(cudaMemcpyAsync(M.xy.p, xy, sizeof(double) * 2 * nv, cudaMemcpyDeviceToDevice, s));
    if (ntri > 0)
        PCMS_CU(cudaMemcpyAsync(M.tri.p, tri, sizeof(int32_t) * 3 * ntri, cudaMemcpyDeviceToDevice, s));
    // bounding box of the vertices
    const int nbb = bbox_blocks(nv);
    DBuf part(sizeof(double) * 8 * nbb, s);
    launch_bbox_partials(2, M.xy.as<double>(), nv, part.as<double>(), s);
    std::vector<double> hp(8 * (size_t)nbb);
    if (nv > 0)
        PCMS_CU(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * 8 * nbb, cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    double hb[6];
    uint64_t hbad = 0;
    bbox_combine(hp.data(), nv, hb, hb + 3, &hbad);
    if (hbad) fail(PCMS_ERR_INVALID_ARG, "non-finite vertex coordinate");
    if (nv == 0) { hb[0] = hb[1] = 0.0; hb[3] = hb[4] = 0.0; }
    M.bbox[0] = hb[0]; M.bbox[1] = hb[1]; M.bbox[2] = hb[3]; M.bbox[3] = hb[4];
    // about one cell per two triangles
    double ex = std::max(hb[3] - hb[0], 0.0), ey = std::max(hb[4] - hb[1], 0.0);
    double area = std::max(ex * ey, 1e-300);
    double h = std::sqrt(area / (0.5 * (double)std::max<int64_t>(ntri, 1)));
    if (!(h > 0.0) || !std::isfinite(h)) h = std::max(std::max(ex, ey), 1.0);
    h = std::max(h, std::max(ex, ey) / 16384.0);
    if (h == 0.0) h = 1.0;
    double lo[3] = {hb[0], hb[1], 0.0}, hi[3] = {hb[3], hb[4], 0.0};
    // make_grid adds the 2^-20 margin used for radius searches; harmless here
    M.g = make_grid(2, lo, hi, h, int64_t(1) << 26);
    const Grid& g = M.g;
    // FP32 orientation filter frame: origin at the box corner, error allowance from the extent
    M.origin[0] = hb[0];
    M.origin[1] = hb[1];
    const double ext = std::max(ex, ey);
    M.use32 = ext > 1e-30 && ext < 1e18;
    M.delta = M.use32 ? (float)(std::ldexp(ext, -44) * (1.0 + 1e-6)) : 0.f;
    M.vhl.alloc(sizeof(float4) * std::max<int64_t>(nv, 1), s);
    if (nv > 0) {
        PCMS_TRACE("mesh_vertex_hilo", s);
        k_vertex_hilo<<<blocks_for(nv, 256), 256, 0, s>>>(nv, M.xy.as<double>(), M.origin[0],
                                                          M.origin[1], M.vhl.as<float4>());
    }
    DBuf count(sizeof(int32_t) * (g.ncell + 1), s);
    PCMS_CU(cudaMemsetAsync(count.p, 0, count.bytes, s));
    M.tsign.alloc(sizeof(int8_t) * std::max<int64_t>(ntri, 1), s);
    DBuf trect(sizeof(int4) * std::max<int64_t>(ntri, 1), s);
    DBuf badid(sizeof(unsigned long long), s);
    PCMS_CU(cudaMemsetAsync(badid.p, 0, badid.bytes, s));
    if (ntri > 0) {
        PCMS_TRACE("mesh_tri_prep", s);
        k_tri_prep<<<blocks_for(ntri, 256), 256, 0, s>>>(nv, M.xy.as<double>(), ntri,
                                                         M.tri.as<int32_t>(), g, count.as<int32_t>(),
                                                         M.tsign.as<int8_t>(), trect.as<int4>(),
                                                         badid.as<unsigned long long>(),
                                                         M.vhl.as<float4>(), M.use32 ? 1 : 0,
                                                         M.delta, (float)g.inv_h);
    }
    PCMS_LAUNCH_CHECK("k_tri_prep");
    M.cell_start.alloc(sizeof(int32_t) * (g.ncell + 1), s);
    exclusive_scan<int32_t>(count.as<int32_t>(), M.cell_start.as<int32_t>(), g.ncell, s);
    int32_t npairs = 0;
    unsigned long long hbadid = 0;
    PCMS_CU(cudaMemcpyAsync(&npairs, M.cell_start.as<int32_t>() + g.ncell, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaMemcpyAsync(&hbadid, badid.p, sizeof(hbadid), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    if (hbadid) fail(PCMS_ERR_INVALID_ARG, "triangle vertex id out of range");
    if (npairs < 0) fail(PCMS_ERR_CAPACITY, "too many (cell, triangle) pairs");
    M.npairs = npairs;
    M.items.alloc(sizeof(int32_t) * std::max<int32_t>(npairs, 1), s);
    PCMS_CU(cudaMemsetAsync(count.p, 0, count.bytes, s));
    if (ntri > 0) {
        PCMS_TRACE("mesh_tri_fill", s);
        k_tri_fill<<<blocks_for(ntri, 256), 256, 0, s>>>(ntri, g, trect.as<int4>(),
                                                         M.cell_start.as<int32_t>(),
                                                         count.as<int32_t>(), M.items.as<int32_t>());
    }
    PCMS_TRACE("mesh_cell_sort", s);
    k_cell_sort<<<blocks_for(g.ncell, 256), 256, 0, s>>>(g.ncell, M.cell_start.as<int32_t>(),
                                                         M.items.as<int32_t>());
    PCMS_LAUNCH_CHECK("mesh build");
}

// ---------------------------------------------------------------------- centroids, P1 integral
__global__ void k_tri_centroid(int64_t nv, const double* __restrict__ xy, int64_t nt,
                               const int32_t* __restrict__ tri, double* __restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = tri[k], b = tri[nt + k], c = tri[2 * nt + k];
        out[k] = __ddiv_rn(__dadd_rn(__dadd_rn(xy[a], xy[b]), xy[c]), 3.0);
        out[nt + k] = __ddiv_rn(__dadd_rn(__dadd_rn(xy[nv + a], xy[nv + b]), xy[nv + c]), 3.0);
    }
}

constexpr int INTEGRAL_THREADS = 256;
constexpr int INTEGRAL_BLOCKS = 1024;

// fixed-order sum of one value per thread over the block (tree in shared memory)
__device__ __forceinline__ double block_sum_fixed(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = INTEGRAL_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    return sh[0];
}

// per-block partial sums of |area| (f0 + f1 + f2) / 3, each thread over a fixed stride
__global__ void __launch_bounds__(INTEGRAL_THREADS) k_tri_integral(
    int64_t nv, const double* __restrict__ xy, int64_t nt, const int32_t* __restrict__ tri,
    const double* __restrict__ f, double* __restrict__ partial) {
    __shared__ double sh[INTEGRAL_THREADS];
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = tri[k], b = tri[nt + k], c = tri[2 * nt + k];
        const double x0 = xy[a], y0 = xy[nv + a];
        const double cr = __dsub_rn(__dmul_rn(__dsub_rn(xy[b], x0), __dsub_rn(xy[nv + c], y0)),
                                    __dmul_rn(__dsub_rn(xy[nv + b], y0), __dsub_rn(xy[c], x0)));
        const double area = __dmul_rn(fabs(cr), 0.5);
        const double mean = __ddiv_rn(__dadd_rn(__dadd_rn(f[a], f[b]), f[c]), 3.0);
        acc = __dadd_rn(acc, __dmul_rn(area, mean));
    }
    const double s = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(INTEGRAL_THREADS) k_sum_partials(const double* __restrict__ partial,
                                                                    int n, double* __restrict__ out) {
    __shared__ double sh[INTEGRAL_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = __dadd_rn(acc, partial[i]);
    const double s = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0) *out = s;
}

void mesh_centroids(const MeshImpl& M, double* out, cudaStream_t s) {
    if (M.ntri <= 0) return;
    PCMS_TRACE("mesh_centroids", s);
    k_tri_centroid<<<blocks_for(M.ntri, 256), 256, 0, s>>>(M.nv, M.xy.as<double>(), M.ntri,
                                                           M.tri.as<int32_t>(), out);
    PCMS_LAUNCH_CHECK("k_tri_centroid");
}

double mesh_integrate(const MeshImpl& M, const double* field, cudaStream_t s) {
    if (M.ntri <= 0) return 0.0;
    const int blocks = (int)std::min<int64_t>(INTEGRAL_BLOCKS, (M.ntri + INTEGRAL_THREADS - 1) / INTEGRAL_THREADS);
    DBuf part(sizeof(double) * (blocks + 1), s);
    {
        PCMS_TRACE("mesh_integrate", s);
        k_tri_integral<<<blocks, INTEGRAL_THREADS, 0, s>>>(M.nv, M.xy.as<double>(), M.ntri,
                                                           M.tri.as<int32_t>(), field,
                                                           part.as<double>());
    }
    {
        PCMS_TRACE("mesh_integrate_sum", s);
        k_sum_partials<<<1, INTEGRAL_THREADS, 0, s>>>(part.as<double>(), blocks,
                                                      part.as<double>() + blocks);
    }
    PCMS_LAUNCH_CHECK("k_tri_integral");
    double h = 0.0;
    PCMS_CU(cudaMemcpyAsync(&h, part.as<double>() + blocks, sizeof(h), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    return h;
}

int64_t estimate_mesh_bytes(int64_t nv, int64_t ntri, int64_t npts) {
    (void)npts;
    // copies of the mesh, orientation signs, rectangles, cell counts/starts, (cell, tri) pairs
    double b = nv * 32.0 + ntri * (12.0 + 1.0 + 16.0) + 2.0 * 4.0 * (0.5 * ntri + 64.0) +
               4.0 * 4.0 * ntri;
    return (int64_t)(1.2 * b) + (int64_t(1) << 20);
}

void mesh_locate(const MeshImpl& M, const double* pts, int64_t n, const double* field,
                 int32_t* elem, int8_t* edim, double* vals, cudaStream_t s) {
    if (n <= 0) return;
    PCMS_TRACE("mesh_locate_interp", s);
    k_locate<<<blocks_for(n, 256), 256, 0, s>>>(
        M.g, M.bbox[0], M.bbox[1], M.bbox[2], M.bbox[3], M.nv, M.xy.as<double>(), M.ntri,
        M.tri.as<int32_t>(), M.tsign.as<int8_t>(), M.cell_start.as<int32_t>(),
        M.items.as<int32_t>(), M.vhl.as<float4>(), M.origin[0], M.origin[1], M.delta, M.use32,
        (float)M.g.inv_h, pts, n, field, elem, edim, vals);
    PCMS_LAUNCH_CHECK("k_locate");
}

}  // namespace pcms
