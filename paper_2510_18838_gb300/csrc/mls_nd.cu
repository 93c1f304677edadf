// mls_nd.cu -- the MLS transfer in four and five dimensions (the paper maps fields in up to
// five dimensions: abstract, and Sec. 5.2's 5D distribution function), in FP64.
//
// The definitions are those of 2D and 3D (Sec. 3.2.1): selection d2 < r^2 with phi > 0,
// d2 summed left to right in FP64 without contraction; per-target (or global) radius
// doubling; weighted normal equations in the target-centred basis scaled by 1/r; guarded
// LDL^T solve; operator rows N_j = w_j a(u_j)^T y; apply by the shared sparse kernels.
// What differs is the search and the split of the work:
//   * a uniform grid in D dimensions with cell edge h >= (r/2)(1 + 2^-20) (doubled until
//     the grid has at most max(2^16, 8 n_src) cells); the box of (2R+1)^D cells around a
//     target, R = floor(r / h) + 1, is walked as (2R+1)^(D-1) rows of cells contiguous in x,
//     and each candidate is screened in FP32 before the exact FP64 test (walk_nd);
//   * one thread per target. The FP64 pipe is the bound (a quadratic basis in 5D has 126
//     moments per pair, 1/64 of the FP32 rate on this GPU), and a thread per target needs no
//     cross-lane reduction of the moments, which would cost more FP64 instructions than the
//     accumulation itself.
// Targets are sorted by cell as in 2D/3D, so neighbouring threads walk neighbouring cells.
#include <algorithm>
#include <cmath>

#include "mls_kernels.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

constexpr int ND_THREADS = 128;

struct GridN {
    int n[ND_MAX_DIM];
    int64_t ncell;
    double lo[ND_MAX_DIM];
    double h, inv_h;
};

GridN make_grid_nd(int D, const double* lo, const double* hi, double radius, int64_t max_cells) {
    GridN g{};
    double h = radius * (1.0 + std::ldexp(1.0, -20));
    for (;;) {
        double tot = 1.0;
        for (int d = 0; d < D; d++) tot *= std::floor((hi[d] - lo[d]) / h) + 1.0;
        if (tot <= (double)max_cells) break;
        h *= 2.0;
    }
    g.ncell = 1;
    for (int d = 0; d < ND_MAX_DIM; d++) {
        g.lo[d] = d < D ? lo[d] : 0.0;
        g.n[d] = d < D ? (int)(std::floor((hi[d] - lo[d]) / h) + 1.0) : 1;
        g.ncell *= g.n[d];
    }
    g.h = h;
    g.inv_h = 1.0 / h;
    return g;
}

__device__ __forceinline__ long long enc_d(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double dec_d(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFLL));
}

// enc[0..D) minima, enc[D..2D) maxima (order-preserving encodings), bad = non-finite count
__global__ void k_bbox_nd_init(int D, long long* enc, unsigned long long* bad) {
    const int i = threadIdx.x;
    if (i < D) enc[i] = 0x7FFFFFFFFFFFFFFFLL;
    else if (i < 2 * D) enc[i] = (long long)0x8000000000000000ULL;
    if (i == 0) *bad = 0;
}

__global__ void k_bbox_nd(int D, const double* __restrict__ pts, int64_t n, long long* enc,
                          unsigned long long* bad) {
    double lo[ND_MAX_DIM], hi[ND_MAX_DIM];
    for (int d = 0; d < ND_MAX_DIM; d++) {
        lo[d] = INFINITY;
        hi[d] = -INFINITY;
    }
    unsigned long long nb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < D; d++) {
            const double x = pts[d * n + i];
            if (!isfinite(x)) {
                nb++;
                continue;
            }
            lo[d] = fmin(lo[d], x);
            hi[d] = fmax(hi[d], x);
        }
    for (int d = 0; d < D; d++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, o);
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < D; d++)
            if (lo[d] <= hi[d]) {
                atomicMin(&enc[d], enc_d(lo[d]));
                atomicMax(&enc[D + d], enc_d(hi[d]));
            }
        if (nb) atomicAdd(bad, nb);
    }
}

__global__ void k_bbox_nd_decode(int D, const long long* enc, double* box) {
    const int i = threadIdx.x;
    if (i < 2 * D) box[i] = dec_d(enc[i]);
}

int grid_blocks(int64_t n, int threads) {
    const int64_t need = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 32));
}

// Bounding box of the sources (lo, hi) after checking both point sets are finite (one sync).
void box_nd(int D, const double* src, int64_t ns, const double* tgt, int64_t nt, double* lo,
            double* hi, cudaStream_t s) {
    DBuf buf(sizeof(long long) * 4 * ND_MAX_DIM + sizeof(unsigned long long) * 2 +
                 sizeof(double) * 2 * ND_MAX_DIM, s);
    long long* enc = buf.as<long long>();
    unsigned long long* bad = (unsigned long long*)(enc + 4 * ND_MAX_DIM);
    double* box = (double*)(bad + 2);
    for (int i = 0; i < 2; i++) {
        PCMS_TRACE("nd_bbox_init", s);
        k_bbox_nd_init<<<1, 32, 0, s>>>(D, enc + 2 * ND_MAX_DIM * i, bad + i);
    }
    for (int i = 0; i < 2; i++) {
        const int64_t n = i == 0 ? ns : nt;
        if (n == 0) continue;
        PCMS_TRACE("nd_bbox_reduce", s);
        k_bbox_nd<<<grid_blocks(n, 256), 256, 0, s>>>(D, i == 0 ? src : tgt, n,
                                                      enc + 2 * ND_MAX_DIM * i, bad + i);
    }
    {
        PCMS_TRACE("nd_bbox_decode", s);
        k_bbox_nd_decode<<<1, 32, 0, s>>>(D, enc, box);
    }
    PCMS_LAUNCH_CHECK("nd_bbox");
    double hb[2 * ND_MAX_DIM];
    unsigned long long hbad[2];
    PCMS_CU(cudaMemcpyAsync(hb, box, sizeof(double) * 2 * D, cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaMemcpyAsync(hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    if (hbad[0] || hbad[1])
        fail(PCMS_ERR_INVALID_ARG, "non-finite point coordinate (" + std::to_string(hbad[0]) +
                                       " in sources, " + std::to_string(hbad[1]) + " in targets)");
    for (int d = 0; d < D; d++) {
        lo[d] = ns > 0 ? hb[d] : 0.0;
        hi[d] = ns > 0 ? hb[D + d] : 0.0;
    }
}

__device__ __forceinline__ int cell_nd(double x, double lo, double inv_h, int n) {
    double f = floor((x - lo) * inv_h);
    f = fmin(fmax(f, 0.0), (double)(n - 1));
    return (int)f;
}

template <int D>
__global__ void k_keys_nd(GridN g, const double* __restrict__ pts, int64_t n,
                          uint32_t* __restrict__ key, uint32_t* __restrict__ idx,
                          int32_t* __restrict__ count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0, stride = 1;
#pragma unroll
        for (int d = 0; d < D; d++) {
            c += stride * cell_nd(pts[d * n + i], g.lo[d], g.inv_h, g.n[d]);
            stride *= g.n[d];
        }
        key[i] = (uint32_t)c;
        idx[i] = (uint32_t)i;
        if (count) atomicAdd(&count[c], 1);
    }
}

// fs[pos] = f[perm[pos]]: a field into the sources' sorted order
__global__ void k_permute_nd(const double* __restrict__ f, const int32_t* __restrict__ perm,
                             int64_t n, double* __restrict__ fs) {
    for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < n;
         pos += (int64_t)gridDim.x * blockDim.x)
        fs[pos] = f[perm[pos]];
}

template <int D>
__global__ void k_gather_nd(GridN g, const double* __restrict__ pts, int64_t n,
                            const uint32_t* __restrict__ order, int32_t* __restrict__ perm,
                            int32_t* __restrict__ inv, double* __restrict__ x64,
                            float* __restrict__ xf) {
    for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < n;
         pos += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = order[pos];
        perm[pos] = (int32_t)i;
        inv[i] = (int32_t)pos;
#pragma unroll
        for (int d = 0; d < D; d++) {
            const double x = pts[d * n + i];
            x64[d * n + pos] = x;
            if (xf) xf[d * n + pos] = (float)(x - g.lo[d]);
        }
    }
}

// points sorted by cell (stable: caller order inside a cell), with cell starts if asked
template <int D>
void sort_nd(const GridN& g, const double* pts, int64_t n, bool with_start, SortedPoints& out,
             cudaStream_t s) {
    out.dim = D;
    out.n = n;
    const int64_t nn = std::max<int64_t>(n, 1);
    out.perm.alloc(sizeof(int32_t) * nn, s);
    out.inv.alloc(sizeof(int32_t) * nn, s);
    out.x64.alloc(sizeof(double) * D * nn, s);
    if (with_start) out.xf.alloc(sizeof(float) * D * nn, s);
    DBuf kv(sizeof(uint32_t) * 4 * nn, s);
    uint32_t* k0 = kv.as<uint32_t>();
    uint32_t* v0 = k0 + nn;
    uint32_t* k1 = v0 + nn;
    uint32_t* v1 = k1 + nn;
    DBuf count;
    if (with_start) {
        count.alloc(sizeof(int32_t) * (g.ncell + 1), s);
        PCMS_CU(cudaMemsetAsync(count.p, 0, count.bytes, s));
        out.cell_start.alloc(sizeof(int32_t) * (g.ncell + 1), s);
    }
    if (n > 0) {
        PCMS_TRACE("nd_cell_keys", s);
        k_keys_nd<D><<<grid_blocks(n, 256), 256, 0, s>>>(g, pts, n, k0, v0,
                                                          with_start ? count.as<int32_t>() : nullptr);
    }
    PCMS_LAUNCH_CHECK("nd_keys");
    if (with_start) exclusive_scan<int32_t>(count.as<int32_t>(), out.cell_start.as<int32_t>(), g.ncell, s);
    if (n > 0) {
        const uint32_t* order = radix_sort_pairs(k0, v0, k1, v1, n, g.ncell, s);
        PCMS_TRACE("nd_gather_sorted", s);
        k_gather_nd<D><<<grid_blocks(n, 256), 256, 0, s>>>(g, pts, n, order, out.perm.as<int32_t>(),
                                                            out.inv.as<int32_t>(), out.x64.as<double>(),
                                                            with_start ? out.xf.as<float>() : nullptr);
    }
    PCMS_LAUNCH_CHECK("nd_gather");
}

struct NdArgs {
    GridN g;
    int64_t ns, nt;
    const int32_t* cell_start;
    const double* sx64;   // [D][ns] sorted sources
    const float* sxf;     // [D][ns] the same as FP32 offsets from the grid origin (filter)
    float src_extent;     // max over d and sources of |s_d - lo_d|
    const double* tx64;   // [D][nt] sorted targets
    RadiusLevels lv;
    int weight;
    int need;
    int32_t* counts;
    int32_t* kexp;        // in: starting/fixed level (assembly); out: doublings (count)
    const int64_t* offsets;
    int32_t* cols;
    const double* field;  // FUSED: sorted field
    double* mom;          // [nt][NACCP]
    double* wvals;        // MAP: each row's weights w_j beside its columns (in the
                          // operator-value buffer, which k_shape_nd overwrites with the rows):
                          // written by the column walk when it assembles the moments, else by
                          // k_moments_nd
};

// Calls f(j, d2) for every source j selected at radius level k of target t (coordinates tt),
// in cell order.
//
// Candidates are first screened in FP32 (most of the box lies outside the ball: the ball
// fills 5.3 r^5 of the (5r)^5 / 32 box in 5D with cells of r/2), and only those that may be
// inside get the exact FP64 test. The screen rejects d2f > r^2 (1 + band), which is sound:
// with the offsets from the grid origin rounded to FP32 (error <= 2^-24 |x - lo| each, so
// <= eta = (ds + dt)(1 + 2^-24) + 2^-24 r per coordinate of s - t near the ball, ds and dt
// the sources' and the target's 2^-24 max |x_d - lo_d|), a source within r has
// sum e_f^2 < (r + sqrt(D) eta)^2 (Minkowski) and d2f <= (1 + D 2^-23)(r + sqrt(D) eta)^2.
// band is that bound relative to r^2, and r2 (1 + band) is rounded up by a further 2^-20.
// The screen is off (band > 1/4) when the FP32 offsets are too coarse for the radius.
//
// The same bound read the other way accepts without the FP64 test: a candidate with
// d2f < r^2 (1 - 2 band) (1 - 2^-20) lies within r (1 - 2^-21), so its FP64 squared distance
// is below r^2 (1 - 2^-40) and it is selected for every weight that is positive on the whole
// support (all but TPS and cubic, which keep the exact test). With NEED_D2 the callback gets
// the FP64 squared distance of every selected pair; without it, d2 is passed only where the
// exact test computed it (0 otherwise).
template <int D, bool NEED_D2 = true, typename F>
__device__ __forceinline__ void walk_nd(const NdArgs& A, const double* tt, int k, F&& f) {
    const GridN& g = A.g;
    const double r = A.lv.r[k], r2 = A.lv.r2[k];
    const double r2_in = r2 * (1.0 - 9.094947017729282e-13);
    const int R = (int)fmin(floor(r * g.inv_h) + 1.0, 1073741824.0);
    float tf[D];
    float tmax = 0.f;
#pragma unroll
    for (int d = 0; d < D; d++) {
        tf[d] = (float)(tt[d] - g.lo[d]);
        tmax = fmaxf(tmax, fabsf(tf[d]));
    }
    float r2hi = INFINITY, r2lo = -1.f;
    if (A.sxf) {
        const float rf = A.lv.r2f[k] > 0.f ? sqrtf(A.lv.r2f[k]) : 0.f;
        const float ds = 5.9604645e-08f * A.src_extent * (1.f + 1e-6f);
        const float dt = 5.9604645e-08f * tmax * (1.f + 1e-6f);
        const float eta = (ds + dt) * (1.f + 5.9604645e-08f) + 5.9604645e-08f * rf;
        const float grow = 1.f + sqrtf((float)D) * eta / rf;
        const float band = (1.f + (float)D * 1.1920929e-07f) * grow * grow - 1.f;
        if (rf > 0.f && band < 0.25f) {
            r2hi = A.lv.r2f[k] * (1.f + band) * (1.f + 9.5367432e-07f);
            if (A.weight != PCMS_TPS && A.weight != PCMS_CUBIC)
                r2lo = A.lv.r2f[k] * (1.f - 2.f * band) * (1.f - 9.5367432e-07f);
        }
    }
    // The box's rows of cells (contiguous in x) are walked in order. A row whose cells lie
    // farther than r from the target in the other D - 1 coordinates is skipped, and the x
    // range of the others is trimmed to the ball's chord at the row's nearest point. Both
    // are computed in cell units in FP32 with a margin mg far above the FP32 error (the
    // positions inside the cell are exact to 2^-24, the cells' own coordinates are exact
    // integers), so they only ever over-cover: every source within r keeps its candidacy.
    int lo_c[D], hi_c[D], idx[D], cc[D];
    float fr[D];
#pragma unroll
    for (int d = 0; d < D; d++) {
        const double p = (tt[d] - g.lo[d]) * g.inv_h;
        double fl = floor(p);
        fl = fmin(fmax(fl, -1073741824.0), 1073741824.0);
        const long long c = (long long)fl;
        cc[d] = (int)c;
        fr[d] = (float)(p - fl);
        lo_c[d] = (int)max(c - R, 0LL);
        hi_c[d] = (int)min(c + R, (long long)g.n[d] - 1);
        if (lo_c[d] > hi_c[d]) return;   // the box misses the grid
        idx[d] = lo_c[d];
    }
    const float R0 = A.lv.rcell[k];
    const float mg = 1e-3f + R0 * 1e-6f;
    const float RR = R0 + mg;
    int64_t stride_c[D];   // cells per step of coordinate d in the linear cell index
    stride_c[0] = 1;
#pragma unroll
    for (int d = 1; d < D; d++) stride_c[d] = stride_c[d - 1] * g.n[d - 1];
    for (;;) {
        // the row's squared distance from the target over the coordinates d >= 1, less mg each
        float rem = RR * RR;
#pragma unroll
        for (int d = 1; d < D; d++) {
            const float dd = (float)(idx[d] - cc[d]);
            float e = fmaxf(fmaxf(dd - fr[d], fr[d] - dd - 1.f), 0.f);
            e = fmaxf(e - mg, 0.f);
            rem -= e * e;
        }
        int x0 = 1, x1 = 0;   // empty unless the row reaches into the ball
        if (rem > 0.f) {
            const float hx = sqrtf(rem) + mg;
            x0 = (int)max((long long)__float2int_rd(fr[0] - hx) + cc[0], (long long)lo_c[0]);
            x1 = (int)min((long long)__float2int_rd(fr[0] + hx) + cc[0], (long long)hi_c[0]);
        }
        int a = 0, b = 0;
        if (x0 <= x1) {
            int64_t base = 0;
#pragma unroll
            for (int d = 1; d < D; d++) base += stride_c[d] * idx[d];
            a = A.cell_start[base + x0];
            b = A.cell_start[base + x1 + 1];
        }
        for (int j = a; j < b; j++) {
            if (A.sxf) {
                float d2f = 0.f;
#pragma unroll
                for (int d = 0; d < D; d++) {
                    const float e = A.sxf[d * A.ns + j] - tf[d];
                    d2f = fmaf(e, e, d2f);
                }
                if (d2f > r2hi) continue;
                if (!NEED_D2 && d2f < r2lo) {
                    f(j, 0.0);
                    continue;
                }
            }
            double e = __dsub_rn(A.sx64[j], tt[0]);
            double d2 = __dmul_rn(e, e);
            e = __dsub_rn(A.sx64[A.ns + j], tt[1]);
            d2 = __dadd_rn(d2, __dmul_rn(e, e));
#pragma unroll
            for (int d = 2; d < D; d++) {
                e = __dsub_rn(A.sx64[d * A.ns + j], tt[d]);
                d2 = __dadd_rn(d2, __dmul_rn(e, e));
            }
            if (select64(A.weight, d2, r, r2, r2_in)) f(j, d2);
        }
        // next row: an odometer over d = 1 .. D-1 with compile-time indices, so that the
        // indices stay in registers
        bool carry = true;
#pragma unroll
        for (int d = 1; d < D; d++) {
            if (carry) {
                if (idx[d] < hi_c[d]) {
                    ++idx[d];
                    carry = false;
                } else {
                    idx[d] = lo_c[d];
                }
            }
        }
        if (carry) break;
    }
}

template <int D>
__device__ __forceinline__ void load_target_nd(const NdArgs& A, int64_t t, double* tt) {
#pragma unroll
    for (int d = 0; d < D; d++) tt[d] = A.tx64[d * A.nt + t];
}

// neighbour counts with per-target growth (need > 0), starting at kexp if given
template <int D>
__global__ void __launch_bounds__(ND_THREADS) k_count_nd(NdArgs A, const int32_t* kstart) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < A.nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        double tt[D];
        load_target_nd<D>(A, t, tt);
        int k = kstart ? kstart[t] : 0;
        int cnt = 0;
        for (;;) {
            cnt = 0;
            walk_nd<D, false>(A, tt, k, [&](int, double) { ++cnt; });
            if (A.need > 0 && cnt < A.need && k < MAX_DOUBLINGS && cnt < A.ns) {
                ++k;
                continue;
            }
            break;
        }
        A.counts[t] = cnt;
        A.kexp[t] = k;
    }
}

__global__ void k_fill_i32(int32_t* v, int64_t n, const unsigned long long* value) {
    const int32_t x = (int32_t)*value;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = x;
}

__global__ void k_max_nd(const int32_t* __restrict__ v, int64_t n, unsigned long long* out) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)max(v[i], 0));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// moments w u^p (degree <= 2 DEG) and, fused, w b u^p (degree <= DEG) of one selected pair
template <int D, int DEG, int MODE, int NACC>
__device__ __forceinline__ void accumulate_nd(double (&acc)[NACC], const double* u, double w,
                                              double b) {
    constexpr int NM = mono_count(D, 2 * DEG);
    constexpr int M = mono_count(D, DEG);
    double wm[NM];
    wm[0] = w;
    acc[0] += w;
    sfor<NM - 1>([&](auto I) {
        constexpr int p = decltype(I)::value + 1;
        constexpr int par = mono_parent_nd<D>(p);
        constexpr int v = mono_var_nd<D>(p);
        wm[p] = wm[par] * u[v];
        acc[p] += wm[p];
    });
    if constexpr (MODE == MODE_FUSED) {
        sfor<M>([&](auto I) {
            constexpr int p = decltype(I)::value;
            acc[NM + p] += wm[p] * b;
        });
    }
}

// operator columns (MAP) and, with MOMENTS, the moments at the target's level kexp[t]
template <int D, int DEG, int MODE, bool MOMENTS = true>
__global__ void __launch_bounds__(ND_THREADS) k_assemble_nd(NdArgs A) {
    constexpr int NM = mono_count(D, 2 * DEG);
    constexpr int M = mono_count(D, DEG);
    constexpr int NACC = MODE == MODE_FUSED ? NM + M : NM;
    constexpr int NACCP = round_up4(NACC);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < A.nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        double tt[D];
        load_target_nd<D>(A, t, tt);
        const int k = A.kexp[t];
        const double inv_r = A.lv.inv_r[k];
        double acc[NACC];
#pragma unroll
        for (int i = 0; i < NACC; i++) acc[i] = 0.0;
        int64_t w_at = MODE == MODE_MAP ? A.offsets[t] : 0;
        const int64_t w_end = MODE == MODE_MAP ? w_at + A.counts[t] : 0;
        walk_nd<D, MOMENTS>(A, tt, k, [&](int j, double d2) {
            double w = 0.0;
            if constexpr (MOMENTS) {
                w = weight_value<double>(A.weight, sqrt(d2) * inv_r);
                double u[D];
#pragma unroll
                for (int d = 0; d < D; d++) u[d] = (A.sx64[d * A.ns + j] - tt[d]) * inv_r;
                accumulate_nd<D, DEG, MODE, NACC>(acc, u, w, MODE == MODE_FUSED ? A.field[j] : 0.0);
            }
            if (MODE == MODE_MAP && w_at < w_end) {
                if (MOMENTS && A.wvals) A.wvals[w_at] = w;   // else k_moments_nd writes it
                A.cols[w_at++] = j;
            }
        });
        if constexpr (MOMENTS) {
            double* dst = A.mom + t * NACCP;
#pragma unroll
            for (int i = 0; i < NACCP; i++) dst[i] = i < NACC ? acc[i < NACC ? i : 0] : 0.0;
        }
    }
}

// The moments of a quadratic basis (degree <= 4) as products of two monomials of degree
// <= 2: moment p = alpha(p) beta(p), alpha = its first min(deg, 2) variable occurrences in
// variable order, beta = the rest. `order` lists the moments grouped by alpha.
template <int D>
struct SplitTab {
    static constexpr int N = MonoTab<D>::N;
    int alpha[N], beta[N], order[N];
};
template <int D>
constexpr SplitTab<D> make_split_tab() {
    SplitTab<D> t{};
    constexpr int N = SplitTab<D>::N;
    for (int p = 0; p < N; ++p) {
        const Exp5 e = mono_exp_nd<D>(p);
        Exp5 ea{}, eb{};
        int seen = 0;
        for (int d = 0; d < D; ++d)
            for (int c = 0; c < e.e[d]; ++c) {
                if (seen < 2) ea.e[d] += 1;
                else eb.e[d] += 1;
                ++seen;
            }
        if (seen <= 2) {   // degree <= 2: the monomial itself times 1
            ea = e;
            eb = Exp5{};
        }
        t.alpha[p] = mono_index_nd<D>(ea);
        t.beta[p] = mono_index_nd<D>(eb);
        t.order[p] = p;
    }
    for (int i = 1; i < N; ++i)   // stable insertion sort by alpha
        for (int k = i; k > 0 && t.alpha[t.order[k - 1]] > t.alpha[t.order[k]]; --k) {
            const int x = t.order[k];
            t.order[k] = t.order[k - 1];
            t.order[k - 1] = x;
        }
    return t;
}

constexpr int ND_REG = 64;   // moments accumulated in registers; the rest in shared memory

// Shared-memory accumulators of k_moments_nd per block: the moments past ND_REG, one double
// per moment and lane ([moment][lane]: a warp's loads and stores hit distinct banks).
template <int D>
constexpr int nd_smem_moments() {
    return mono_count(D, 4) > ND_REG ? mono_count(D, 4) - ND_REG : 0;
}
template <int D>
constexpr size_t nd_moments_smem_bytes() {
    return sizeof(double) * (size_t)nd_smem_moments<D>() * ND_THREADS;
}

// Moments of a quadratic basis from the operator's row, in one pass over it. The 126 (5D)
// accumulators do not fit one thread's registers: ND_REG of them are registers, the others
// live in shared memory, one slot per lane (a load, a multiply-add and a store per pair).
// The shared-memory traffic runs beside the FP64 pipe, the bound, which then carries each
// pair's offsets, weight and monomials once. A warp per target: its lanes take the row's
// pairs 32 apart (rows of uneven length cost a warp only their own length, where a thread per
// target made each warp wait for its longest row), and the lanes' partial sums are added by a
// butterfly of shuffles at the end (5 adds per moment, against one multiply-add per moment
// and pair). Per pair: the offsets and the squared distance as the walk's exact test forms
// them, the weight (kept in the operator-value buffer, where the rows find it), the degree
// <= 2 monomials a2 of u, then for each moment one FMA, (w a2[alpha]) a2[beta], with
// w a2[alpha] formed once per alpha group.
template <int D>
__global__ void __launch_bounds__(ND_THREADS) k_moments_nd(NdArgs A) {
    constexpr int NM = mono_count(D, 4);
    constexpr int M2 = mono_count(D, 2);
    constexpr int NACCP = round_up4(NM);
    constexpr int NR = NM < ND_REG ? NM : ND_REG;
    constexpr int NS = nd_smem_moments<D>();
    constexpr SplitTab<D> tab = make_split_tab<D>();
    extern __shared__ double nd_sacc[];
    const int lane = threadIdx.x & 31;
    volatile double* sacc = nd_sacc + (threadIdx.x >> 5) * 32 * NS + lane;   // [NS][32]
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < A.nt;
         t += nwarps) {
        double tt[D];
        load_target_nd<D>(A, t, tt);
        const int k = A.kexp[t];
        const double inv_r = A.lv.inv_r[k];
        const int64_t a = A.offsets[t], b = a + A.counts[t];
        double* dst = A.mom + t * NACCP;
        double acc[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) acc[q] = 0.0;
#pragma unroll
        for (int q = 0; q < NS; q++) sacc[32 * q] = 0.0;
        for (int64_t i = a + lane; i < b; i += 32) {
            const int j = A.cols[i];
            double u[D];
            double e = __dsub_rn(A.sx64[j], tt[0]);
            double d2 = __dmul_rn(e, e);
            u[0] = e * inv_r;
#pragma unroll
            for (int d = 1; d < D; d++) {
                e = __dsub_rn(A.sx64[d * A.ns + j], tt[d]);
                d2 = __dadd_rn(d2, __dmul_rn(e, e));
                u[d] = e * inv_r;
            }
            const double w = weight_value<double>(A.weight, sqrt(d2) * inv_r);
            A.wvals[i] = w;
            double a2[M2];
            a2[0] = 1.0;
            sfor<M2 - 1>([&](auto I) {
                constexpr int p = decltype(I)::value + 1;
                constexpr int par = mono_parent_nd<D>(p);
                constexpr int v = mono_var_nd<D>(p);
                a2[p] = a2[par] * u[v];
            });
            double wa = 0.0;
            sfor<NM>([&](auto Q) {
                constexpr int q = decltype(Q)::value;
                constexpr int p = tab.order[q];
                constexpr int al = tab.alpha[p];
                constexpr int be = tab.beta[p];
                constexpr bool fresh = q == 0 || tab.alpha[tab.order[q - 1]] != al;
                if constexpr (fresh) wa = w * a2[al];
                if constexpr (q < NR) acc[q] = fma(wa, a2[be], acc[q]);
                else sacc[32 * (q - NR)] = fma(wa, a2[be], sacc[32 * (q - NR)]);
            });
        }
        sfor<NM>([&](auto Q) {
            constexpr int q = decltype(Q)::value;
            double v;
            if constexpr (q < NR) v = acc[q];
            else v = sacc[32 * (q - NR)];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == (q & 31)) dst[tab.order[q]] = v;
        });
        if (lane < NACCP - NM) dst[NM + lane] = 0.0;
    }
}

struct NdSolveArgs {
    int64_t nt;
    const int32_t* counts;
    const double* mom;
    double lambda;
    double* y;              // MAP: [nt][m]
    int8_t* status;         // MAP: sorted order; FUSED: caller order via perm_t
    const int32_t* perm_t;
    double* out;            // FUSED: caller-order values
};

template <int D, int DEG, int MODE>
__global__ void __launch_bounds__(ND_THREADS) k_solve_nd(NdSolveArgs S) {
    constexpr int NM = mono_count(D, 2 * DEG);
    constexpr int M = mono_count(D, DEG);
    constexpr int NACC = MODE == MODE_FUSED ? NM + M : NM;
    constexpr int NACCP = round_up4(NACC);
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < S.nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        int st = PCMS_TARGET_OK;
        double y[M], val = 0.0, amp = 0.0;
        if (S.counts[t] < M) {
            st = PCMS_TARGET_UNDERDETERMINED;
        } else {
            double mom[NACC];
#pragma unroll
            for (int i = 0; i < NACC; i++) mom[i] = S.mom[t * NACCP + i];
            if (!solve_moments<D, DEG, MODE>(mom, S.lambda, 1e-14, y, &val, &amp, nullptr))
                st = PCMS_TARGET_ILL_CONDITIONED;
        }
        if (MODE == MODE_FUSED) {
            const int64_t o = S.perm_t[t];
            S.out[o] = st == PCMS_TARGET_OK ? val : nanv;
            if (S.status) S.status[o] = (int8_t)st;
        } else {
#pragma unroll
            for (int i = 0; i < M; i++) S.y[t * M + i] = st == PCMS_TARGET_OK ? y[i] : nanv;
            S.status[t] = (int8_t)st;
        }
    }
}

// operator rows N_j = w_j a(u_j)^T y, with w_j as the column walk wrote it into vals (the
// same buffer); a warp per target, its lanes over the row's pairs 32 apart
template <int D, int DEG>
__global__ void __launch_bounds__(ND_THREADS) k_shape_nd(NdArgs A, const double* __restrict__ yv,
                                                         double* __restrict__ vals) {
    constexpr int M = mono_count(D, DEG);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < A.nt;
         t += nwarps) {
        double tt[D], y[M];
        load_target_nd<D>(A, t, tt);
#pragma unroll
        for (int i = 0; i < M; i++) y[i] = yv[t * M + i];
        const int k = A.kexp[t];
        const double inv_r = A.lv.inv_r[k];
        const int64_t a = A.offsets[t], b = a + A.counts[t];
        for (int64_t i = a + lane; i < b; i += 32) {
            const int j = A.cols[i];
            const double w = vals[i];
            double u[D];
#pragma unroll
            for (int d = 0; d < D; d++) u[d] = __dsub_rn(A.sx64[d * A.ns + j], tt[d]) * inv_r;
            double am[M];
            am[0] = 1.0;
            double s = y[0];
            sfor<M - 1>([&](auto I) {
                constexpr int p = decltype(I)::value + 1;
                constexpr int par = mono_parent_nd<D>(p);
                constexpr int v = mono_var_nd<D>(p);
                am[p] = am[par] * u[v];
                s += am[p] * y[p];
            });
            vals[i] = w * s;
        }
    }
}

// out: [0] underdetermined, [1] ill-conditioned, [2] max count, [3] max doublings, [4] nnz
__global__ void k_stats_nd(const int8_t* status, const int32_t* counts, const int32_t* kexp,
                           int64_t n, unsigned long long* out) {
    unsigned long long under = 0, ill = 0, mc = 0, mk = 0, sc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        under += status[i] == PCMS_TARGET_UNDERDETERMINED;
        ill += status[i] == PCMS_TARGET_ILL_CONDITIONED;
        mc = max(mc, (unsigned long long)counts[i]);
        mk = max(mk, (unsigned long long)kexp[i]);
        sc += (unsigned long long)counts[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        under += __shfl_xor_sync(0xffffffffu, under, o);
        ill += __shfl_xor_sync(0xffffffffu, ill, o);
        mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], under);
        atomicAdd(&out[1], ill);
        atomicMax(&out[2], mc);
        atomicMax(&out[3], mk);
        atomicAdd(&out[4], sc);
    }
}

__global__ void k_counts_to_caller_nd(int64_t nt, const int32_t* __restrict__ perm_t,
                                      const int32_t* __restrict__ c, const int32_t* __restrict__ k,
                                      int32_t* __restrict__ c_out, int32_t* __restrict__ k_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        c_out[perm_t[i]] = c[i];
        if (k_out) k_out[perm_t[i]] = k[i];
    }
}

int nd_blocks(int64_t n) { return grid_blocks(n, ND_THREADS); }

// The search state shared by the entry points: sorted points, grid, counts and doublings
// (per target, or the global reading), for dimension D.
template <int D>
struct NdSearch {
    GridN g;
    NdArgs a;
};

template <int D>
NdSearch<D> search_nd(const MlsParams& P, const double* src, int64_t ns, const double* tgt,
                      int64_t nt, SortedPoints& S, SortedPoints& T, DBuf& counts, DBuf& kexp,
                      cudaStream_t s) {
    double lo[ND_MAX_DIM], hi[ND_MAX_DIM];
    box_nd(D, src, ns, tgt, nt, lo, hi, s);
    NdSearch<D> r;
    r.g = make_grid_nd(D, lo, hi, 0.5 * P.radius,
                       std::min<int64_t>(int64_t(1) << 26, std::max<int64_t>(int64_t(1) << 16, 8 * ns)));
    sort_nd<D>(r.g, src, ns, true, S, s);
    sort_nd<D>(r.g, tgt, nt, false, T, s);
    counts.alloc(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    kexp.alloc(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    NdArgs& a = r.a;
    a = NdArgs{};
    a.g = r.g;
    a.ns = ns;
    a.nt = nt;
    a.cell_start = S.cell_start.as<int32_t>();
    a.sx64 = S.x64.as<double>();
    a.sxf = S.xf.as<float>();
    {
        double ext = 0.0;
        for (int d = 0; d < D; d++) ext = std::max(ext, std::max(std::fabs(hi[d] - lo[d]), 0.0));
        a.src_extent = (float)(ext * (1.0 + 1e-6));
    }
    a.tx64 = T.x64.as<double>();
    a.lv = make_radius_levels(P.radius, r.g.inv_h);
    a.weight = (int)P.weight;
    a.need = P.need;
    a.counts = counts.as<int32_t>();
    a.kexp = kexp.as<int32_t>();
    if (nt > 0) {
        {
            PCMS_TRACE("nd_count", s);
            k_count_nd<D><<<nd_blocks(nt), ND_THREADS, 0, s>>>(a, nullptr);
        }
        PCMS_LAUNCH_CHECK("nd_count");
        if (P.need > 0 && P.growth == PCMS_GROWTH_GLOBAL) {
            // one shared radius: the largest per-target doubling (counts grow with r)
            DBuf mx(sizeof(unsigned long long), s);
            PCMS_CU(cudaMemsetAsync(mx.p, 0, mx.bytes, s));
            {
                PCMS_TRACE("nd_global_doublings", s);
                k_max_nd<<<nd_blocks(nt), ND_THREADS, 0, s>>>(a.kexp, nt, mx.as<unsigned long long>());
            }
            {
                PCMS_TRACE("nd_global_fill", s);
                k_fill_i32<<<nd_blocks(nt), ND_THREADS, 0, s>>>(a.kexp, nt, mx.as<unsigned long long>());
            }
            NdArgs b = a;
            b.need = 0;
            PCMS_TRACE("nd_count", s);
            k_count_nd<D><<<nd_blocks(nt), ND_THREADS, 0, s>>>(b, a.kexp);
            PCMS_LAUNCH_CHECK("nd_global");
        }
    }
    a.need = 0;   // the levels are fixed from here on
    return r;
}

template <int D, int DEG>
void create_map_nd(MapImpl& M, const double* src, const double* tgt) {
    cudaStream_t s = M.stream;
    const MlsParams& P = M.P;
    constexpr int M_ = mono_count(D, DEG);
    constexpr int NACCP = round_up4(mono_count(D, 2 * DEG));
    const int64_t ns = M.ns, nt = M.nt;
    NdSearch<D> r = search_nd<D>(P, src, ns, tgt, nt, M.src, M.tgt, M.counts, M.kexp, s);
    NdArgs a = r.a;
    M.status.alloc(sizeof(int8_t) * std::max<int64_t>(nt, 1), s);
    M.offsets.alloc(sizeof(int64_t) * (nt + 1), s);
    exclusive_scan<int64_t>(M.counts.as<int32_t>(), M.offsets.as<int64_t>(), nt, s);
    int64_t nnz = 0;
    PCMS_CU(cudaMemcpyAsync(&nnz, M.offsets.as<int64_t>() + nt, sizeof(nnz), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    M.nnz = nnz;
    M.cols.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1), s);
    M.vals.alloc(sizeof(double) * std::max<int64_t>(nnz, 1), s);
    if (nt > 0) {
        DBuf mom(sizeof(double) * NACCP * nt, s);
        DBuf y(sizeof(double) * M_ * nt, s);
        a.offsets = M.offsets.as<int64_t>();
        a.cols = M.cols.as<int32_t>();
        a.mom = mom.as<double>();
        a.wvals = M.vals.as<double>();   // the rows' weights until k_shape_nd replaces them
        if constexpr (DEG == 2) {   // columns first, then the moments in passes over the rows
            {
                PCMS_TRACE("nd_assemble_map", s);
                k_assemble_nd<D, DEG, MODE_MAP, false><<<nd_blocks(nt), ND_THREADS, 0, s>>>(a);
            }
            {
                PCMS_TRACE("nd_moments", s);
                constexpr size_t smem = nd_moments_smem_bytes<D>();
                if (smem > 48 * 1024)
                    PCMS_CU(cudaFuncSetAttribute(k_moments_nd<D>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
                k_moments_nd<D><<<nd_blocks(32 * nt), ND_THREADS, smem, s>>>(a);   // warp per target
            }
        } else {
            PCMS_TRACE("nd_assemble_map", s);
            k_assemble_nd<D, DEG, MODE_MAP><<<nd_blocks(nt), ND_THREADS, 0, s>>>(a);
        }
        PCMS_LAUNCH_CHECK("nd_assemble");
        NdSolveArgs sa{};
        sa.nt = nt;
        sa.counts = M.counts.as<int32_t>();
        sa.mom = mom.as<double>();
        sa.lambda = P.lambda;
        sa.y = y.as<double>();
        sa.status = M.status.as<int8_t>();
        {
            PCMS_TRACE("nd_solve_map", s);
            k_solve_nd<D, DEG, MODE_MAP><<<nd_blocks(nt), ND_THREADS, 0, s>>>(sa);
        }
        PCMS_LAUNCH_CHECK("nd_solve");
        {
            PCMS_TRACE("nd_shape", s);
            k_shape_nd<D, DEG><<<nd_blocks(32 * nt), ND_THREADS, 0, s>>>(a, y.as<double>(),
                                                                     M.vals.as<double>());
        }
        PCMS_LAUNCH_CHECK("nd_shape");
        DBuf st(sizeof(unsigned long long) * 5, s);
        PCMS_CU(cudaMemsetAsync(st.p, 0, st.bytes, s));
        {
            PCMS_TRACE("nd_status_stats", s);
            k_stats_nd<<<nd_blocks(nt), ND_THREADS, 0, s>>>(M.status.as<int8_t>(), M.counts.as<int32_t>(),
                                                           M.kexp.as<int32_t>(), nt,
                                                           st.as<unsigned long long>());
        }
        PCMS_LAUNCH_CHECK("nd_stats");
        unsigned long long hs[5];
        PCMS_CU(cudaMemcpyAsync(hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
        M.n_under = (int64_t)hs[0];
        M.n_ill = (int64_t)hs[1];
        M.max_count = (int64_t)hs[2];
        M.max_k = (int64_t)hs[3];
    }
}

template <int D, int DEG>
void transfer_nd(const MlsParams& P, const double* src, int64_t ns, const double* tgt, int64_t nt,
                 const double* fields, int nf, double* out, int8_t* status, cudaStream_t s,
                 int64_t* n_under) {
    constexpr int NACCP = round_up4(mono_count(D, 2 * DEG) + mono_count(D, DEG));
    SortedPoints S, T;
    DBuf counts, kexp;
    NdSearch<D> r = search_nd<D>(P, src, ns, tgt, nt, S, T, counts, kexp, s);
    NdArgs a = r.a;
    DBuf fs(sizeof(double) * std::max<int64_t>(ns, 1), s);
    DBuf mom(sizeof(double) * NACCP * std::max<int64_t>(nt, 1), s);
    DBuf st(sizeof(unsigned long long) * 5, s);
    PCMS_CU(cudaMemsetAsync(st.p, 0, st.bytes, s));
    for (int f = 0; f < nf && nt > 0; f++) {
        if (ns > 0) {
            PCMS_TRACE("nd_field_to_sorted", s);
            k_permute_nd<<<grid_blocks(ns, 256), 256, 0, s>>>(fields + (int64_t)f * ns,
                                                              S.perm.as<int32_t>(), ns, fs.as<double>());
        }
        a.field = fs.as<double>();
        a.mom = mom.as<double>();
        {
            PCMS_TRACE("nd_assemble_fused", s);
            k_assemble_nd<D, DEG, MODE_FUSED><<<nd_blocks(nt), ND_THREADS, 0, s>>>(a);
        }
        NdSolveArgs sa{};
        sa.nt = nt;
        sa.counts = counts.as<int32_t>();
        sa.mom = mom.as<double>();
        sa.lambda = P.lambda;
        sa.status = f == 0 ? status : nullptr;
        sa.perm_t = T.perm.as<int32_t>();
        sa.out = out + (int64_t)f * nt;
        {
            PCMS_TRACE("nd_solve_fused", s);
            k_solve_nd<D, DEG, MODE_FUSED><<<nd_blocks(nt), ND_THREADS, 0, s>>>(sa);
        }
        PCMS_LAUNCH_CHECK("nd_fused");
    }
    *n_under = 0;
    if (status && P.min_neighbors == 0 && nt > 0) {
        {
            PCMS_TRACE("nd_status_stats", s);
            k_stats_nd<<<nd_blocks(nt), ND_THREADS, 0, s>>>(status, counts.as<int32_t>(),
                                                           kexp.as<int32_t>(), nt,
                                                           st.as<unsigned long long>());
        }
        PCMS_LAUNCH_CHECK("nd_stats");
        unsigned long long hs[5];
        PCMS_CU(cudaMemcpyAsync(hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
        *n_under = (int64_t)hs[0];
    }
}

template <int D>
void count_nd(const MlsParams& P, const double* src, int64_t ns, const double* tgt, int64_t nt,
              int32_t* counts, int32_t* kexp, int64_t* total, cudaStream_t s) {
    SortedPoints S, T;
    DBuf c, k;
    search_nd<D>(P, src, ns, tgt, nt, S, T, c, k, s);
    if (nt > 0) {
        PCMS_TRACE("nd_counts_to_caller", s);
        k_counts_to_caller_nd<<<nd_blocks(nt), ND_THREADS, 0, s>>>(nt, T.perm.as<int32_t>(),
                                                                    c.as<int32_t>(), k.as<int32_t>(),
                                                                    counts, kexp);
        PCMS_LAUNCH_CHECK("nd_counts_to_caller");
    }
    if (total) {
        DBuf off(sizeof(int64_t) * (nt + 1), s);
        exclusive_scan<int64_t>(c.as<int32_t>(), off.as<int64_t>(), nt, s);
        PCMS_CU(cudaMemcpyAsync(total, off.as<int64_t>() + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
    }
}

}  // namespace

void mls_nd_create_map(MapImpl& M, const double* src, const double* tgt) {
    const int D = M.P.dim, deg = M.P.degree;
#define PCMS_ND_MAP(DV, KV) if (D == DV && deg == KV) return create_map_nd<DV, KV>(M, src, tgt)
    PCMS_ND_MAP(4, 0); PCMS_ND_MAP(4, 1); PCMS_ND_MAP(4, 2);
    PCMS_ND_MAP(5, 0); PCMS_ND_MAP(5, 1); PCMS_ND_MAP(5, 2);
#undef PCMS_ND_MAP
    fail(PCMS_ERR_INVALID_ARG, "MLS above 3D: dim must be 4 or 5");
}

void mls_nd_transfer(const MlsParams& P, const double* src, int64_t ns, const double* tgt,
                     int64_t nt, const double* fields, int nf, double* out, int8_t* status,
                     cudaStream_t s, int64_t* n_under) {
    const int D = P.dim, deg = P.degree;
    if (deg == 2) {
        // quadratic: through a transient operator (its moments are accumulated in passes
        // over the rows, which needs the rows)
        MapImpl M;
        M.P = P;
        M.ns = ns;
        M.nt = nt;
        M.stream = s;
        mls_nd_create_map(M, src, tgt);
        mls_apply(M, fields, nf, out, s);
        if (status) mls_export(M, nullptr, nullptr, nullptr, status, nullptr, s);
        *n_under = P.min_neighbors == 0 ? M.n_under : 0;
        return;
    }
#define PCMS_ND_TR(DV, KV) \
    if (D == DV && deg == KV) return transfer_nd<DV, KV>(P, src, ns, tgt, nt, fields, nf, out, status, s, n_under)
    PCMS_ND_TR(4, 0); PCMS_ND_TR(4, 1);
    PCMS_ND_TR(5, 0); PCMS_ND_TR(5, 1);
#undef PCMS_ND_TR
    fail(PCMS_ERR_INVALID_ARG, "MLS above 3D: dim must be 4 or 5");
}

void mls_nd_count(const MlsParams& P, const double* src, int64_t ns, const double* tgt, int64_t nt,
                  int32_t* counts, int32_t* kexp, int64_t* total, cudaStream_t s) {
    if (P.dim == 4) return count_nd<4>(P, src, ns, tgt, nt, counts, kexp, total, s);
    if (P.dim == 5) return count_nd<5>(P, src, ns, tgt, nt, counts, kexp, total, s);
    fail(PCMS_ERR_INVALID_ARG, "MLS above 3D: dim must be 4 or 5");
}

}  // namespace pcms
