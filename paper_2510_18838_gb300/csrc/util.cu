// util.cu -- errors, device memory, bounding box, prefix scan and the counting sort of
// points into uniform-grid cells (the search structure of Sec. 3.3).
#include <climits>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "pcms_internal.cuh"
#include "trace.cuh"

namespace pcms {

void fail(pcms_status st, const std::string& msg) { throw PcmsError{st, msg}; }

void check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    (void)cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? PCMS_ERR_OUT_OF_MEMORY : PCMS_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
}

void ensure_mempool(int device) {
    // Keep freed stream-ordered memory cached in this process's default pool, so that
    // repeated calls do not return memory to the driver at every synchronisation.
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    (void)cudaGetLastError();
    done[device] = true;
}

void DBuf::alloc(size_t b, cudaStream_t st) {
    release();
    s = st;
    bytes = b;
    if (b == 0) return;
    cudaError_t e = cudaMallocAsync(&p, b, st);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        (void)cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? PCMS_ERR_OUT_OF_MEMORY : PCMS_ERR_CUDA,
             std::string("cudaMallocAsync(") + std::to_string(b) + " bytes): " +
                 cudaGetErrorString(e));
    }
}

void DBuf::release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
}

int num_sms() {
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int n = 0;
    PCMS_CU(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}

static double grid_cells(int dim, const double* lo, const double* hi, double h, int xs) {
    double tot = 1.0;
    for (int d = 0; d < dim; d++)
        tot *= std::floor((hi[d] - lo[d]) / h * (d == 0 ? xs : 1)) + 1.0;
    return tot;
}

Grid make_grid(int dim, const double* lo, const double* hi, double radius, int64_t max_cells,
               int xs) {
    Grid g;
    g.dim = dim;
    g.xs = dim >= 2 ? xs : 1;
    double h = radius * (1.0 + std::ldexp(1.0, -20));
    for (int d = 0; d < 3; d++) {
        g.lo[d] = d < dim ? lo[d] : 0.0;
        g.n[d] = 1;
    }
    while (grid_cells(dim, lo, hi, h, g.xs) > (double)max_cells) h *= 2.0;
    int64_t ncell = 1;
    for (int d = 0; d < dim; d++) {
        g.n[d] = (int)(std::floor((hi[d] - lo[d]) / h * (d == 0 ? g.xs : 1)) + 1.0);
        ncell *= g.n[d];
    }
    g.ncell = ncell;
    g.h = h;
    g.inv_h = 1.0 / h;
    return g;
}

int choose_xs(int dim, const double* lo, const double* hi, double cell, int64_t max_cells,
              int64_t ns) {
    if (dim < 2) return 1;
    const double h = cell * (1.0 + std::ldexp(1.0, -20));
    const double cap = (double)std::min<int64_t>(max_cells, 2 * ns + 64);
    for (int xs = 4; xs > 1; xs >>= 1)
        if (grid_cells(dim, lo, hi, h, xs) <= cap) return xs;
    return 1;
}

// ------------------------------------------------------------------------------------
// bounding box
// ------------------------------------------------------------------------------------
// Per-block boxes: block b writes part[8 b + {0..2}] = minima, [3..5] = maxima, [6] = the
// number of non-finite coordinates it saw. One launch, no initialisation; the host combines
// the partial boxes after its copy (bbox_combine). Each thread loads BB_UNROLL points per
// coordinate plane before it reduces them, so that enough loads are in flight for the
// kernel to stream at HBM speed with one block per SM. The comparisons run on the integer
// pipe: a double's bits x map to the signed integer x ^ ((x >> 63) & 0x7fff...), which orders
// like the values (-0 just below +0), so min and max need no FP64 instruction; a coordinate
// is non-finite when its exponent bits are all set.
constexpr int BB_UNROLL = 4;

__device__ __forceinline__ long long order_key(long long b) {
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

template <int DIM>
__global__ void __launch_bounds__(256) k_bbox_partial(const double* __restrict__ pts, int64_t n,
                                                      double* __restrict__ part) {
    __shared__ double sh[8][7];
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    int nb = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const long long* bits = reinterpret_cast<const long long*>(pts);
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n;
         i0 += BB_UNROLL * stride) {
        long long x[DIM][BB_UNROLL];
#pragma unroll
        for (int d = 0; d < DIM; d++)
#pragma unroll
            for (int u = 0; u < BB_UNROLL; u++) {
                const int64_t i = i0 + u * stride;
                x[d][u] = i < n ? bits[d * n + i] : 0LL;
            }
#pragma unroll
        for (int u = 0; u < BB_UNROLL; u++) {
            if (i0 + u * stride >= n) break;
#pragma unroll
            for (int d = 0; d < DIM; d++) {
                const long long b = x[d][u];
                if ((b & 0x7ff0000000000000LL) == 0x7ff0000000000000LL) {
                    nb++;
                    continue;
                }
                const long long k = order_key(b);
                lo[d] = min(lo[d], k);
                hi[d] = max(hi[d], k);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int d = 0; d < 3; d++) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 3; d++) {
            // back to doubles; no finite coordinate on an axis gives (+inf, -inf)
            sh[w][d] = lo[d] == LLONG_MAX ? INFINITY : __longlong_as_double(order_key(lo[d]));
            sh[w][3 + d] = hi[d] == LLONG_MIN ? -INFINITY : __longlong_as_double(order_key(hi[d]));
        }
        sh[w][6] = (double)nb;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int j = 1; j < (int)(blockDim.x >> 5); j++)
            v = k < 3 ? fmin(v, sh[j][k]) : (k < 6 ? fmax(v, sh[j][k]) : v + sh[j][k]);
        part[8 * blockIdx.x + k] = v;
    }
}

int bbox_blocks(int64_t n) {
    const int64_t per_block = 256 * BB_UNROLL;
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block,
                                                       (int64_t)num_sms()));
}

void launch_bbox_partials(int dim, const double* pts, int64_t n, double* part, cudaStream_t s) {
    if (n <= 0) return;
    if (dim < 1 || dim > 3) fail(PCMS_ERR_INVALID_ARG, "internal: bounding box of dim > 3");
    PCMS_TRACE("bbox_partial", s);
    const int nb = bbox_blocks(n);
    if (dim == 1) k_bbox_partial<1><<<nb, 256, 0, s>>>(pts, n, part);
    else if (dim == 2) k_bbox_partial<2><<<nb, 256, 0, s>>>(pts, n, part);
    else k_bbox_partial<3><<<nb, 256, 0, s>>>(pts, n, part);
    PCMS_LAUNCH_CHECK("bbox_partial");
}

void bbox_combine(const double* hpart, int64_t n, double* lo, double* hi, uint64_t* bad) {
    for (int d = 0; d < 3; d++) {
        lo[d] = INFINITY;
        hi[d] = -INFINITY;
    }
    double nb = 0.0;
    if (n > 0)
        for (int b = 0; b < bbox_blocks(n); b++) {
            for (int d = 0; d < 3; d++) {
                lo[d] = std::fmin(lo[d], hpart[8 * b + d]);
                hi[d] = std::fmax(hi[d], hpart[8 * b + 3 + d]);
            }
            nb += hpart[8 * b + 6];
        }
    *bad = (uint64_t)nb;
}

// ------------------------------------------------------------------------------------
// exclusive scan: per-tile reduce -> scan of tile sums -> per-tile scan with offset
// (no inter-block waiting)
// ------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T t = lane < (SCAN_THREADS / 32) ? warp_tot[lane] : T(0);
        T u = t;
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        if (lane < (SCAN_THREADS / 32)) warp_tot[lane] = u - t;
        if (lane == 31) *total = u;
    }
    __syncthreads();
    return x - v + warp_tot[wid];
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t* __restrict__ in,
                                                              int64_t n, T* bsum) {
    __shared__ T wt[SCAN_THREADS / 32];
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++)
        if (base + k < n) s += (T)in[base + k];
    block_exclusive_scan<T>(s, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_bsum(T* bsum, int64_t nb, T* total_out) {
    __shared__ T wt[32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        T v = i < nb ? bsum[i] : T(0);
        T x = v;
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wt[wid] = x;
        __syncthreads();
        if (wid == 0) {
            T t = wt[lane];
            T u = t;
            for (int o = 1; o < 32; o <<= 1) {
                T y = __shfl_up_sync(0xffffffffu, u, o);
                if (lane >= o) u += y;
            }
            wt[lane] = u - t;
        }
        __syncthreads();
        T excl = x - v + wt[wid] + carry;
        if (i < nb) bsum[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const int32_t* __restrict__ in,
                                                            int64_t n, const T* bsum, T* out) {
    __shared__ T wt[SCAN_THREADS / 32];
    __shared__ T tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = base + k < n ? (T)in[base + k] : T(0);
        s += v[k];
    }
    T run = block_exclusive_scan<T>(s, wt, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// Small inputs in one block (one launch instead of three): 1024 threads scan tiles of
// 1024 x SCAN_ITEMS entries in order, carrying the running total.
constexpr int SCAN1_THREADS = 1024;
constexpr int64_t SCAN1_MAX = 32768;

template <typename T>
__global__ void __launch_bounds__(SCAN1_THREADS) k_scan_single(const int32_t* __restrict__ in,
                                                              int64_t n, T* __restrict__ out) {
    __shared__ T wt[32];
    __shared__ T carry_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += (int64_t)SCAN1_THREADS * SCAN_ITEMS) {
        const int64_t i0 = base + (int64_t)threadIdx.x * SCAN_ITEMS;
        T v[SCAN_ITEMS];
        T sum = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; k++) {
            v[k] = i0 + k < n ? (T)in[i0 + k] : T(0);
            sum += v[k];
        }
        T x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wt[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const T t = wt[lane];
            T u = t;
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(0xffffffffu, u, o);
                if (lane >= o) u += y;
            }
            wt[lane] = u - t;
        }
        __syncthreads();
        T run = carry_s + wt[wid] + (x - sum);
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; k++) {
            if (i0 + k < n) out[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == SCAN1_THREADS - 1) carry_s = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry_s;
}

template <typename T>
void exclusive_scan(const int32_t* in, T* out, int64_t n, cudaStream_t s) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 0) {
        PCMS_CU(cudaMemsetAsync(out, 0, sizeof(T), s));
        return;
    }
    if (n <= SCAN1_MAX) {   // also in place: a tile is read before any of it is written
        PCMS_TRACE("scan_single", s);
        k_scan_single<T><<<1, SCAN1_THREADS, 0, s>>>(in, n, out);
        PCMS_LAUNCH_CHECK("scan_single");
        return;
    }
    DBuf bs(sizeof(T) * nb, s);
    {
        PCMS_TRACE("scan_reduce", s);
        k_scan_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bs.as<T>());
    }
    {
        PCMS_TRACE("scan_tile_sums", s);
        k_scan_bsum<T><<<1, 1024, 0, s>>>(bs.as<T>(), nb, out + n);
    }
    {
        PCMS_TRACE("scan_down", s);
        k_scan_down<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bs.as<T>(), out);
    }
    PCMS_LAUNCH_CHECK("exclusive_scan");
}

template void exclusive_scan<int32_t>(const int32_t*, int32_t*, int64_t, cudaStream_t);
template void exclusive_scan<int64_t>(const int32_t*, int64_t*, int64_t, cudaStream_t);

// ------------------------------------------------------------------------------------
// binning points into cells: cell key per point, then a stable LSD radix sort of
// (key, caller index) with 8-bit digits. Stability makes the order inside a cell the caller's
// index order, so everything computed from the sorted points is bitwise reproducible.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ int cell_of(double x, double lo, double inv_h, int n) {
    double f = floor((x - lo) * inv_h);
    f = fmin(fmax(f, 0.0), (double)(n - 1));   // NaN -> 0 (fmax/fmin drop NaN)
    return (int)f;
}

__global__ void k_cell_keys(Grid g, const double* __restrict__ pts, int64_t n,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c = cell_of(pts[i], g.lo[0], g.inv_hd(0), g.n[0]);
        if (g.dim >= 2) c += g.n[0] * cell_of(pts[n + i], g.lo[1], g.inv_h, g.n[1]);
        if (g.dim == 3)
            c += g.n[0] * g.n[1] * cell_of(pts[2 * n + i], g.lo[2], g.inv_h, g.n[2]);
        key[i] = (uint32_t)c;
        idx[i] = (uint32_t)i;
    }
}

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

// per-tile digit histogram, digit-major: hist[d * ntiles + tile]
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t* __restrict__ key,
                                                        int64_t n, int shift, int64_t ntiles,
                                                        int32_t* __restrict__ hist) {
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        const int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// stable scatter: items of a tile are placed in index order within each digit
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           int64_t n, int shift, int64_t ntiles,
                                                           const int32_t* __restrict__ off,
                                                           uint32_t* __restrict__ kout,
                                                           uint32_t* __restrict__ vout) {
    __shared__ int32_t base[256];
    __shared__ int32_t tot[256];
    __shared__ int32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    base[tid] = off[(int64_t)tid * ntiles + blockIdx.x];
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
#pragma unroll
        for (int k = 0; k < RS_THREADS / 32; k++) wcnt[k][tid] = 0;
        __syncthreads();
        const int64_t i = t0 + r * RS_THREADS + tid;
        const bool valid = i < n;
        const uint32_t kv = valid ? kin[i] : 0u;
        const int d = valid ? (int)((kv >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {
            int run = 0;
#pragma unroll
            for (int k = 0; k < RS_THREADS / 32; k++) {
                const int c = wcnt[k][tid];
                wcnt[k][tid] = run;
                run += c;
            }
            tot[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const int pos = base[d] + wcnt[w][d] + rank;
            kout[pos] = kv;
            vout[pos] = vin[i];
        }
        __syncthreads();
        base[tid] += tot[tid];
    }
}

__global__ void k_gather_sorted(int dim, Grid g, const double* __restrict__ pts, int64_t n,
                                const uint32_t* __restrict__ order, int32_t* __restrict__ perm,
                                int32_t* __restrict__ inv, double* __restrict__ x64,
                                float4* __restrict__ hl0, float2* __restrict__ hl1,
                                int4* __restrict__ cell, float4* __restrict__ frac) {
    for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < n;
         pos += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = order[pos];
        perm[pos] = (int32_t)i;
        inv[i] = (int32_t)pos;
        double x[3] = {0, 0, 0};
        for (int d = 0; d < dim; d++) {
            x[d] = pts[d * n + i];
            x64[d * n + pos] = x[d];
        }
        if (cell) point_cell(g, dim, x, &cell[pos], &frac[pos]);
        if (hl0) {
            float h[3], l[3];
            for (int d = 0; d < 3; d++) {
                double rel = x[d] - g.lo[d];
                h[d] = (float)rel;
                l[d] = (float)(rel - (double)h[d]);
            }
            if (dim == 2) {
                hl0[pos] = make_float4(h[0], h[1], l[0], l[1]);
            } else {
                hl0[pos] = make_float4(h[0], h[1], h[2], l[0]);
                hl1[pos] = make_float2(l[1], l[2]);
            }
        }
    }
}

// one warp per h-wide cell (xs adjacent x cells of the grid, contiguous in the sorted
// order): lanes take the cell's sources in strides of 32, then a fixed butterfly reduction
__global__ void k_cell_sums(int dim, int64_t ncell, int nx, int xs, const int32_t* __restrict__ start,
                            const float4* __restrict__ hl0, float4* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int ncx = (nx + xs - 1) / xs;
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncell;
         c += nwarps) {
        const int64_t row = c / ncx;
        const int cx = (int)(c - row * ncx);
        const int64_t base = row * nx;
        const int a = start[base + (int64_t)cx * xs], b = start[base + min((cx + 1) * xs, nx)];
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int i = a + lane; i < b; i += 32) {
            const float4 h = hl0[i];
            sx += h.x;
            sy += h.y;
            if (dim == 3) sz += h.z;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        if (lane == 0) out[c] = make_float4(sx, sy, sz, (float)(b - a));
    }
}

// level j + 1 from level j: each block sums its (up to) 2^dim children in a fixed order
__global__ void k_pyr_up(int dim, int64_t nx, int64_t ny, int64_t nz, int64_t mx, int64_t my,
                         int64_t mz, const float4* __restrict__ in, float4* __restrict__ out) {
    const int64_t nout = mx * my * mz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nout;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bx = i % mx, byz = i / mx, by = byz % my, bz = byz / my;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < (1 << dim); c++) {
            const int64_t x = 2 * bx + (c & 1), y = 2 * by + ((c >> 1) & 1),
                          z = 2 * bz + ((c >> 2) & 1);
            if (x >= nx || y >= ny || z >= nz) continue;
            const float4 v = in[(z * ny + y) * nx + x];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        out[i] = acc;
    }
}

// The pyramid is built over h-wide cells (xs x cells merged).
int pyramid_levels(const Grid& g) {
    int64_t m = std::max<int64_t>(g.ncoarse_x(), std::max<int64_t>(g.n[1], g.n[2]));
    int L = 1;
    while (L < PYR_MAX && m > 1) {
        m = (m + 1) / 2;
        L++;
    }
    return L;
}

int64_t pyramid_size(const Grid& g, int levels, int64_t* off) {
    int64_t n[3] = {g.ncoarse_x(), g.n[1], g.n[2]}, tot = 0;
    for (int j = 0; j < levels; j++) {
        if (off) off[j] = tot;
        tot += n[0] * n[1] * n[2];
        for (int d = 0; d < g.dim; d++) n[d] = (n[d] + 1) / 2;
    }
    return tot;
}

void cell_pyramid(const Grid& g, const SortedPoints& S, int levels, const int64_t* off,
                  float4* out, cudaStream_t s) {
    if (g.ncell <= 0) return;
    PCMS_TRACE("grid_cell_pyramid", s);
    const int64_t ncoarse = g.ncell / g.n[0] * g.ncoarse_x();
    const int64_t blocks = std::min<int64_t>((ncoarse + 7) / 8, (int64_t)num_sms() * 16);
    k_cell_sums<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(
        g.dim, ncoarse, g.n[0], g.xs, S.cell_start.as<int32_t>(), S.hl0.as<float4>(), out);
    int64_t n[3] = {g.ncoarse_x(), g.n[1], g.n[2]};
    for (int j = 1; j < levels; j++) {
        int64_t m[3] = {n[0], n[1], n[2]};
        for (int d = 0; d < g.dim; d++) m[d] = (n[d] + 1) / 2;
        const int64_t nout = m[0] * m[1] * m[2];
        k_pyr_up<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nout + 255) / 256, 4096)), 256, 0,
                   s>>>(g.dim, n[0], n[1], n[2], m[0], m[1], m[2], out + off[j - 1], out + off[j]);
        for (int d = 0; d < 3; d++) n[d] = m[d];
    }
    PCMS_LAUNCH_CHECK("cell_pyramid");
}

uint32_t* radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n,
                           int64_t nkeys, cudaStream_t s, uint32_t** keys_out) {
    if (keys_out) *keys_out = k0;
    if (n <= 0) return v0;
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) < nkeys) bits++;
    const int passes = (bits + 7) / 8;
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    DBuf hist(sizeof(int32_t) * (256 * ntiles + 1), s);
    for (int p = 0; p < passes; p++) {
        {
            PCMS_TRACE("grid_radix_hist", s);
            k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(k0, n, 8 * p, ntiles, hist.as<int32_t>());
        }
        exclusive_scan<int32_t>(hist.as<int32_t>(), hist.as<int32_t>(), 256 * ntiles, s);
        {
            PCMS_TRACE("grid_radix_scatter", s);
            k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(k0, v0, n, 8 * p, ntiles,
                                                                 hist.as<int32_t>(), k1, v1);
        }
        PCMS_LAUNCH_CHECK("radix");
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    if (keys_out) *keys_out = k0;
    return v0;
}

// cell_start[c] = the first sorted position whose key is >= c, for c = 0..ncell. Position
// pos writes the cells (key[pos - 1], key[pos]] (position n: the cells after the last key),
// so every entry is written exactly once, without atomics.
__global__ void k_cell_starts(const uint32_t* __restrict__ skey, int64_t n, int64_t ncell,
                              int32_t* __restrict__ start) {
    for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos <= n;
         pos += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = pos == 0 ? 0 : (int64_t)skey[pos - 1] + 1;
        const int64_t hi = pos == n ? ncell : (int64_t)skey[pos];
        for (int64_t c = lo; c <= hi; c++) start[c] = (int32_t)pos;
    }
}

// The same by a binary search per cell, for grids with many more cells than points (long
// runs of empty cells would serialise the kernel above).
__global__ void k_cell_starts_search(const uint32_t* __restrict__ skey, int64_t n, int64_t ncell,
                                     int32_t* __restrict__ start) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = 0, b = n;   // first position in [a, b) with key >= c
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if ((int64_t)skey[m] < c) a = m + 1;
            else b = m;
        }
        start[c] = (int32_t)a;
    }
}

void sort_points(const Grid& g, const double* pts, int64_t n, bool with_start, bool with_hl,
                 SortedPoints& out, cudaStream_t s, bool with_cell) {
    out.dim = g.dim;
    out.n = n;
    const int dim = g.dim;
    const int64_t nn = std::max<int64_t>(n, 1);
    // cell starts only where they are needed (sources); targets are only ordered
    DBuf kv(sizeof(uint32_t) * 4 * nn, s);   // key, idx, key', idx'
    uint32_t* k0 = kv.as<uint32_t>();
    uint32_t* v0 = k0 + nn;
    uint32_t* k1 = v0 + nn;
    uint32_t* v1 = k1 + nn;
    out.perm.alloc(sizeof(int32_t) * nn, s);
    out.inv.alloc(sizeof(int32_t) * nn, s);
    out.x64.alloc(sizeof(double) * dim * nn, s);
    if (with_hl) {
        out.hl0.alloc(sizeof(float4) * nn, s);
        if (dim == 3) out.hl1.alloc(sizeof(float2) * nn, s);
    }
    if (with_cell) {
        out.cell.alloc(sizeof(int4) * nn, s);
        out.frac.alloc(sizeof(float4) * nn, s);
    }
    if (with_start) out.cell_start.alloc(sizeof(int32_t) * (g.ncell + 1), s);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
    if (n > 0) {
        PCMS_TRACE("grid_cell_keys", s);
        k_cell_keys<<<blocks, 256, 0, s>>>(g, pts, n, k0, v0);
    }
    PCMS_LAUNCH_CHECK("cell_keys");
    uint32_t* skey = k0;
    if (n > 0) v0 = radix_sort_pairs(k0, v0, k1, v1, n, g.ncell, s, &skey);
    if (with_start) {
        PCMS_TRACE("grid_cell_starts", s);
        if (g.ncell <= 8 * n)
            k_cell_starts<<<(int)std::max<int64_t>(1, std::min<int64_t>((n + 256) / 256, (int64_t)num_sms() * 8)),
                            256, 0, s>>>(skey, n, g.ncell, out.cell_start.as<int32_t>());
        else
            k_cell_starts_search<<<(int)std::max<int64_t>(1, std::min<int64_t>((g.ncell + 256) / 256, (int64_t)num_sms() * 8)),
                                   256, 0, s>>>(skey, n, g.ncell, out.cell_start.as<int32_t>());
        PCMS_LAUNCH_CHECK("cell_starts");
    }
    if (n > 0) {
        PCMS_TRACE("grid_gather_sorted", s);
        k_gather_sorted<<<blocks, 256, 0, s>>>(dim, g, pts, n, v0, out.perm.as<int32_t>(),
                                               out.inv.as<int32_t>(), out.x64.as<double>(),
                                               with_hl ? out.hl0.as<float4>() : nullptr,
                                               (with_hl && dim == 3) ? out.hl1.as<float2>() : nullptr,
                                               with_cell ? out.cell.as<int4>() : nullptr,
                                               with_cell ? out.frac.as<float4>() : nullptr);
    }
    PCMS_LAUNCH_CHECK("gather_sorted");
}

}  // namespace pcms
