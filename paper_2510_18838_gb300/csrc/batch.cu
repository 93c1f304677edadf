// batch.cu -- batched one-shot MLS transfer of many small, independent problems
// (Sec. 3.2.1, Eq. 1: one local weighted least-squares fit per target, independent across
// targets and across problems), for the serving loop and for callers with many small
// transfers (pcms_mls_transfer_batch).
//
// A small transfer run through the general path costs tens of launches and several host
// syncs (bounding box, radix-sort passes, scans, precision tiers, status counts) for very
// little arithmetic. Here a batch of problems of one shape class (dimension, basis degree,
// lanes per target) costs two kernels, replayed as one CUDA graph:
//
//   k_batch_sort   one thread block per problem: bounding box and finiteness check of its
//                  points, its uniform grid (cell edge r/3 in 2D, r/2 in 3D, doubled until
//                  the cells fit the problem's cell budget), cell keys, a counting sort with
//                  the sources of each cell put back in index order (so the order does not
//                  depend on atomics), sorted FP64 coordinates and FP32 hi/lo offsets from
//                  the grid origin, and the fields in sorted order, [n_src][fp].
//   k_batch_mls    persistent over (problem, tile of targets) work units taken from a
//                  counter, so that problems with uneven neighbour counts share the GPU.
//                  Per target, a group of G lanes walks the candidate rows (as k_assemble
//                  does), classifies each candidate in FP32 and decides the 2^-16 band
//                  around r^2 exactly in FP64, and stages the selected sources in shared
//                  memory. From the stage it accumulates the FP32 moments, solves them
//                  (refined FP32 LDL^T, FP64 on decline) and checks the conditioning estimate
//                  amp against the plain tier's bound; a rejected target is assembled and
//                  solved again in FP64 in the same kernel. Then every selected source's
//                  operator row value N_j = w_j a(u_j)^T y is applied to all fields at once.
//
// All sizes are bounded on the host from the problem sizes, so nothing is read back between
// the kernels; per-problem errors (a non-finite coordinate) come back in the batch header.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "mls_kernels.cuh"
#include "pcms_batch.cuh"
#include "qr.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

constexpr int SORT_THREADS = 1024;
constexpr int MLS_THREADS = 256;
// guard thresholds, as the general path's: plain FP32 pivots below TAU32 G_kk go to the
// FP64 assembly; the FP64 guard is the definition's rank test (R_kk^2 <= 1e-14 ||B_k||^2)
constexpr double TAU32 = 1e-5;
constexpr double TAU64 = 1e-14;
// FP64 normal equations give c_0 to about amp / rho 2^-53 (rho the smallest LDL^T pivot
// ratio): fits through about m nearly degenerate points lose more than the mixed path's
// bound (the normal equations square the condition number of the weighted Vandermonde
// matrix). Targets whose amp / rho stays above AMP_QR after the re-centred pass are solved
// again by Householder QR of that matrix, whose error grows with its condition number only.
// At most QR_MAX neighbours (such fits are small).
constexpr double AMP_QR = AMP_QR_MIXED;
constexpr int QR_WARPS = 4;

template <int G>
struct BatchShape {
    static constexpr int GPW = 32 / G;                    // targets per warp
    static constexpr int TILE = (MLS_THREADS / 32) * GPW;  // targets per work unit
    static constexpr int STG = G == 32 ? 1024 : 256;      // staged sources per target
};

__device__ __forceinline__ double ordered_min(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double ordered_max(double a, double b) { return a > b ? a : b; }

// block-wide reduction of per-thread values; op 0 = min, 1 = max, 2 = or (as double)
__device__ __forceinline__ double block_reduce(double v, int op, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double x = __shfl_xor_sync(0xffffffffu, v, o);
        v = op == 0 ? ordered_min(v, x) : (op == 1 ? ordered_max(v, x) : (v != 0.0 || x != 0.0 ? 1.0 : 0.0));
    }
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? sh[lane] : (op == 0 ? INFINITY : (op == 1 ? -INFINITY : 0.0));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double x = __shfl_xor_sync(0xffffffffu, v, o);
            v = op == 0 ? ordered_min(v, x) : (op == 1 ? ordered_max(v, x) : (v != 0.0 || x != 0.0 ? 1.0 : 0.0));
        }
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    return sh[32];
}

// exclusive scan in place of a[0..n) (int32, total below 2^31) by one block
__device__ void block_exclusive_scan(int32_t* a, int64_t n, int32_t* sh) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int64_t chunk = (n + nt - 1) / nt;
    const int64_t b0 = min((int64_t)tid * chunk, n), b1 = min(b0 + chunk, n);
    int32_t s = 0;
    for (int64_t i = b0; i < b1; i++) s += a[i];
    // scan of the per-thread sums
    const int lane = tid & 31, w = tid >> 5;
    int32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    __syncthreads();
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t v = lane < (nt >> 5) ? sh[lane] : 0;
        int32_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t x = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += x;
        }
        sh[lane] = vi - v;   // exclusive prefix of the warp sums
    }
    __syncthreads();
    int32_t run = sh[w] + incl - s;
    for (int64_t i = b0; i < b1; i++) {
        const int32_t c = a[i];
        a[i] = run;
        run += c;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------
// k_batch_sort: one block per problem (blocks loop over the problems)
// ------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(SORT_THREADS) k_batch_sort(BatchHeader* hdr, BatchReq* reqs) {
    __shared__ double shd[33];
    __shared__ int32_t shi[32];
    __shared__ double g_lo[3];
    __shared__ double g_inv_h;
    __shared__ int g_n[3];
    __shared__ int g_bad;
    const int n_req = hdr->n_req;
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // k_batch_mls's work counter, the QR list
        hdr->next = 0;
        hdr->n_qr = 0;
    }
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int r = blockIdx.x; r < n_req; r += gridDim.x) {
        BatchReq* q = reqs + r;
        const int64_t ns = q->ns, nt = q->nt;
        const double* src = q->src;
        const double* tgt = q->tgt;
        // 1. bounding box of the sources; finiteness of every coordinate
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double bad = 0.0;
        for (int64_t i = tid; i < ns; i += nth) {
#pragma unroll
            for (int d = 0; d < DIM; d++) {
                const double x = src[d * ns + i];
                if (!isfinite(x)) bad = 1.0;
                lo[d] = fmin(lo[d], x);
                hi[d] = fmax(hi[d], x);
            }
        }
        for (int64_t i = tid; i < nt; i += nth) {
#pragma unroll
            for (int d = 0; d < DIM; d++)
                if (!isfinite(tgt[d * nt + i])) bad = 1.0;
        }
        bad = block_reduce(bad, 2, shd);
        for (int d = 0; d < DIM; d++) {
            lo[d] = block_reduce(lo[d], 0, shd);
            hi[d] = block_reduce(hi[d], 1, shd);
        }
        // 2. the grid: cell edge r/3 (2D) or r/2 (3D), doubled until it fits the budget
        if (tid == 0) {
            g_bad = bad != 0.0;
            hdr->err[r] = g_bad;
        }
        __syncthreads();
        if (g_bad) continue;
        if (tid == 0) {
            double h = DIM == 2 ? q->radius / 3.0 : q->radius / 2.0;
            int n[3] = {1, 1, 1};
            for (int it = 0; it < 200; it++) {
                double tot = 1.0;
                for (int d = 0; d < DIM; d++) {
                    const double e = ns > 0 ? hi[d] - lo[d] : 0.0;
                    const double c = floor(e / h) + 1.0;
                    n[d] = (int)fmin(c, 1073741824.0);
                    tot *= c;
                }
                if (tot <= (double)q->cap_cells) break;
                h *= 2.0;
            }
            for (int d = 0; d < 3; d++) {
                g_lo[d] = (d < DIM && ns > 0) ? lo[d] : 0.0;
                g_n[d] = d < DIM ? n[d] : 1;
                q->lo[d] = g_lo[d];
                q->n[d] = g_n[d];
            }
            g_inv_h = 1.0 / h;
            q->h = h;
            q->inv_h = g_inv_h;
            q->rcell = (float)fmin(q->radius * g_inv_h, 1073741824.0);
        }
        __syncthreads();
        const int64_t ncell = (int64_t)g_n[0] * g_n[1] * g_n[2];
        int32_t* cs = q->cell_start;
        int32_t* cur = q->cursor;
        int32_t* keys = q->keys;
        int32_t* perm = q->perm;
        // 3. counts per cell
        for (int64_t c = tid; c <= ncell; c += nth) cs[c] = 0;
        __syncthreads();
        for (int64_t i = tid; i < ns; i += nth) {
            int64_t key = 0;
#pragma unroll
            for (int d = DIM - 1; d >= 0; d--) {
                const double u = (src[d * ns + i] - g_lo[d]) * g_inv_h;
                const int c = (int)fmin(fmax(floor(u), 0.0), (double)(g_n[d] - 1));
                key = key * g_n[d] + c;
            }
            keys[i] = (int32_t)key;
            atomicAdd(&cs[key], 1);
        }
        __syncthreads();
        // 4. cell starts (cs[ncell] = ns), cursors
        block_exclusive_scan(cs, ncell + 1, shi);
        for (int64_t c = tid; c < ncell; c += nth) cur[c] = cs[c];
        __syncthreads();
        // 5. scatter, then each cell's sources in ascending index order
        for (int64_t i = tid; i < ns; i += nth) perm[atomicAdd(&cur[keys[i]], 1)] = (int32_t)i;
        __syncthreads();
        for (int64_t c = tid; c < ncell; c += nth) {
            const int32_t a = cs[c], b = cs[c + 1];
            for (int32_t x = a + 1; x < b; x++) {
                const int32_t v = perm[x];
                int32_t y = x - 1;
                while (y >= a && perm[y] > v) {
                    perm[y + 1] = perm[y];
                    y--;
                }
                perm[y + 1] = v;
            }
        }
        __syncthreads();
        // 6. sorted coordinates (FP64, FP32 hi/lo offsets from the origin) and fields
        const int nf = q->nf, fp = q->fp;
        for (int64_t p = tid; p < ns; p += nth) {
            const int64_t j = perm[p];
            float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int d = 0; d < DIM; d++) {
                const double x = src[d * ns + j];
                q->x64[d * ns + p] = x;
                const double off = x - g_lo[d];
                h[d] = (float)off;
                l[d] = (float)(off - (double)h[d]);
            }
            if (DIM == 2) {
                q->hl0[p] = make_float4(h[0], h[1], l[0], l[1]);
            } else {
                q->hl0[p] = make_float4(h[0], h[1], h[2], l[0]);
                q->hl1[p] = make_float2(l[1], l[2]);
            }
            if (fp == 1) {
                q->fs[p] = q->fields[j];
            } else {
                float4* row = reinterpret_cast<float4*>(q->fs + p * fp);
                for (int v = 0; v < fp / 4; v++) {
                    float t4[4];
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const int f = 4 * v + c;
                        t4[c] = f < nf ? q->fields[(int64_t)f * ns + j] : 0.f;
                    }
                    row[v] = make_float4(t4[0], t4[1], t4[2], t4[3]);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// k_batch_mls
// ------------------------------------------------------------------------------------
// FP32 offsets of sorted source j from the target, from the hi/lo pairs
template <int DIM>
__device__ __forceinline__ void offsets32(const BatchReq& R, int j, const float* thi,
                                          const float* tlo, float* dx) {
    const float4 a = R.hl0[j];
    if (DIM == 2) {
        dx[0] = (a.x - thi[0]) + (a.z - tlo[0]);
        dx[1] = (a.y - thi[1]) + (a.w - tlo[1]);
        dx[2] = 0.f;
    } else {
        const float2 b = R.hl1[j];
        dx[0] = (a.x - thi[0]) + (a.w - tlo[0]);
        dx[1] = (a.y - thi[1]) + (b.x - tlo[1]);
        dx[2] = (a.z - thi[2]) + (b.y - tlo[2]);
    }
}

// Walk of one target's candidate rows by a group of G lanes (the row set-up, chords and
// candidate stream of k_assemble). Selected sources (sorted positions) are appended to the
// group's stage; when fewer than G free entries remain, flush(n) is called on the staged
// entries and the stage restarts (*spilled). Returns the number of selected sources; the
// last *staged entries are left in the stage.
template <int DIM, int G, class Flush>
__device__ __forceinline__ int walk_select(const BatchReq& R, const Grid& g, const long long* ct,
                                           const float* fr, const float* thi, const float* tlo,
                                           const double* tx, int* rA, int* rE, int32_t* stg,
                                           int stg_cap, int gl, unsigned gmask, int& staged,
                                           bool& spilled, Flush&& flush) {
    const float R0 = R.rcell;
    const float mg = 1e-3f + R0 * 1e-6f;
    const float RR = R0 + mg;
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    long long z0 = 0, z1 = 0;
    if (DIM == 3) {
        z0 = max((long long)__float2int_rd(fr[2] - RR), -ct[2]);
        z1 = min((long long)__float2int_rd(fr[2] + RR), (long long)g.n[2] - 1 - ct[2]);
    }
    const long long y0 = max((long long)__float2int_rd(fr[1] - RR), -ct[1]);
    const long long y1 = min((long long)__float2int_rd(fr[1] + RR), (long long)g.n[1] - 1 - ct[1]);
    const long long ny = y1 >= y0 ? y1 - y0 + 1 : 0;
    const long long nrows = ny * (DIM == 3 ? (z1 >= z0 ? z1 - z0 + 1 : 0) : 1);
    int cnt = 0;
    staged = 0;
    spilled = false;
    for (long long row0 = 0; row0 < nrows; row0 += G) {
        int ra = 0, rlen = 0;
        const long long rho = row0 + gl;
        int64_t rowbase;
        long long x0, x1;
        if (rho < nrows && row_chord<DIM>(g, ct, fr, RR, mg, y0, z0, ny, rho, rowbase, x0, x1)) {
            ra = R.cell_start[rowbase + x0];
            rlen = R.cell_start[rowbase + x1 + 1] - ra;
        }
        int incl = rlen;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const int v = __shfl_up_sync(gmask, incl, o, G);
            if (gl >= o) incl += v;
        }
        const int total = __shfl_sync(gmask, incl, G - 1, G);
        rA[gl] = ra;
        rE[gl] = incl;
        __syncwarp(gmask);
        int rcur = 0;
        for (int p0 = 0; p0 < total; p0 += G) {
            const int p = p0 + gl;
            bool in = false;
            int j = 0;
            if (p < total) {
                while (rE[rcur] <= p) ++rcur;
                j = rA[rcur] + (p - (rcur ? rE[rcur - 1] : 0));
                float dx[3];
                offsets32<DIM>(R, j, thi, tlo, dx);
                float d2f = dx[0] * dx[0] + dx[1] * dx[1];
                if (DIM == 3) d2f += dx[2] * dx[2];
                int cl = classify32(R.weight, d2f, R.r2f);
                if (cl < 0) cl = select_exact(R.weight, dist2_exact<DIM>(R.x64, R.ns, j, tx), R.radius, R.r2);
                in = cl != 0;
            }
            const unsigned bal = __ballot_sync(gmask, in) & gmask;
            if (in) stg[staged + __popc(bal & lt)] = j;
            staged += __popc(bal);
            cnt += __popc(bal);
            __syncwarp(gmask);
            if (staged > stg_cap - G) {
                flush(staged);
                staged = 0;
                spilled = true;
                __syncwarp(gmask);
            }
        }
        __syncwarp(gmask);   // the row table is rewritten by the next G rows
    }
    return cnt;
}

// o[f] += nj fs[j][f] for the fp padded fields of sorted source j (T = float or double)
template <typename T>
__device__ __forceinline__ void apply_row(const BatchReq& R, int j, T nj, T (&o)[16]) {
    if (R.fp == 1) {
        o[0] = fma(nj, (T)R.fs[j], o[0]);
        return;
    }
    const float4* row = reinterpret_cast<const float4*>(R.fs + (int64_t)j * R.fp);
#pragma unroll
    for (int v = 0; v < 4; v++) {
        if (4 * v < R.fp) {
            const float4 x = row[v];
            o[4 * v + 0] = fma(nj, (T)x.x, o[4 * v + 0]);
            o[4 * v + 1] = fma(nj, (T)x.y, o[4 * v + 1]);
            o[4 * v + 2] = fma(nj, (T)x.z, o[4 * v + 2]);
            o[4 * v + 3] = fma(nj, (T)x.w, o[4 * v + 3]);
        }
    }
}

// sums of the group's lanes; lane f % G writes field f of target t (caller order)
template <int G, typename T>
__device__ __forceinline__ void finish_rows(const BatchReq& R, T (&o)[16], int64_t t, int gl,
                                            unsigned gmask) {
#pragma unroll
    for (int f = 0; f < 16; f++) {
        if (f < R.fp) {
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) o[f] += __shfl_xor_sync(gmask, o[f], off);
        }
    }
#pragma unroll
    for (int f = 0; f < 16; f++)
        if (f < R.nf && (f % G) == gl) R.out[(int64_t)f * R.nt + t] = (float)o[f];
}

// Two blocks per SM (128 registers), except the 3D quadratic form: its FP64 fallback
// (35 moments and the 55-entry LDL^T factor in FP64) spills heavily at that size.
template <int DIM, int DEG>
constexpr int batch_min_blocks() {
    return DIM == 3 && DEG == 2 ? 1 : 2;
}

template <int DIM, int DEG, int G>
__global__ void __launch_bounds__(MLS_THREADS, batch_min_blocks<DIM, DEG>()) k_batch_mls(BatchHeader* hdr, const BatchReq* reqs) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    using S = BatchShape<G>;
    constexpr int GPW = S::GPW, TILE = S::TILE, STG = S::STG;
    __shared__ int32_t stg_s[(MLS_THREADS / 32) * GPW * STG];
    __shared__ int rowa_s[MLS_THREADS / 32][32], rowe_s[MLS_THREADS / 32][32];
    __shared__ BatchReq R;
    __shared__ long long item_s;
    __shared__ int req_s;

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gi = lane / G, gl = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
    int32_t* stg = &stg_s[(wib * GPW + gi) * STG];
    int* rA = &rowa_s[wib][gi * G];
    int* rE = &rowe_s[wib][gi * G];
    const int n_req = hdr->n_req;
    const long long total = hdr->total_tiles;
    int cur = -1;
    for (;;) {
        __syncthreads();   // every thread is done with the previous unit's R
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(&hdr->next, 1ull);
            int r = -1;
            if (it < total) {   // the last problem whose first tile is at or before it
                int a = 0, b = n_req - 1;
                while (a < b) {
                    const int mid = (a + b + 1) >> 1;
                    if (reqs[mid].tile0 <= it) a = mid;
                    else b = mid - 1;
                }
                r = a;
            }
            item_s = it;
            req_s = r;
        }
        __syncthreads();
        const long long it = item_s;
        if (it >= total) break;
        const int r = req_s;
        if (r != cur) {
            const int* srcw = reinterpret_cast<const int*>(reqs + r);
            int* dstw = reinterpret_cast<int*>(&R);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchReq) / sizeof(int)); w += blockDim.x)
                dstw[w] = srcw[w];
            cur = r;
            __syncthreads();
        }
        if (hdr->err[r]) continue;
        const int64_t t = (it - R.tile0) * TILE + wib * GPW + gi;
        if (t >= R.nt) continue;

        Grid g;
        g.dim = DIM;
        g.n[0] = R.n[0];
        g.n[1] = R.n[1];
        g.n[2] = R.n[2];
        g.ncell = (int64_t)R.n[0] * R.n[1] * R.n[2];
        g.lo[0] = R.lo[0];
        g.lo[1] = R.lo[1];
        g.lo[2] = R.lo[2];
        g.h = R.h;
        g.inv_h = R.inv_h;
        // the target: FP64 coordinates, FP32 hi/lo offsets from the origin, cell and position
        double tx[3] = {0.0, 0.0, 0.0};
        float thi[3] = {0.f, 0.f, 0.f}, tlo[3] = {0.f, 0.f, 0.f}, fr[3] = {0.f, 0.f, 0.f};
        long long ct[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            tx[d] = R.tgt[d * R.nt + t];
            const double off = tx[d] - g.lo[d];
            thi[d] = (float)off;
            tlo[d] = (float)(off - (double)thi[d]);
            const double u = off * g.inv_h;
            const double fl = fmin(fmax(floor(u), -1073741824.0), 1073741824.0);
            ct[d] = (long long)fl;
            fr[d] = (float)(u - fl);
        }

        // walk 1: FP32 moments of the selected sources
        float acc[NM];
#pragma unroll
        for (int i = 0; i < NM; i++) acc[i] = 0.f;
        auto moments32 = [&](int n) {
            for (int e0 = 0; e0 < n; e0 += G) {
                const int e = e0 + gl;
                if (e < n) {
                    float dx[3];
                    offsets32<DIM>(R, stg[e], thi, tlo, dx);
                    accumulate<DIM, DEG, MODE_MAP, float, NM>(acc, dx, 0.f, R.weight, R.inv_rf, nullptr);
                }
            }
        };
        int staged = 0;
        bool spilled = false;
        const int cnt = walk_select<DIM, G>(R, g, ct, fr, thi, tlo, tx, rA, rE, stg, STG, gl, gmask,
                                            staged, spilled, moments32);
        moments32(staged);   // the last chunk; the stage keeps its entries
        const bool have_all = !spilled;
#pragma unroll
        for (int i = 0; i < NM; i++) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(gmask, acc[i], o);
        }

        // solve (every lane of the group, redundantly: the same inputs, the same path)
        int st = PCMS_TARGET_OK;
        bool fp64 = false, rows64 = false, recentred = false;
        float4 rbasis = make_float4(0.f, 0.f, 0.f, 1.f);   // basis of y64 when recentred
        float yh[M], yl[M];
        double y64[M];
        if (cnt < M) {
            st = PCMS_TARGET_UNDERDETERMINED;
        } else {
            const float bound = amp_bound(ACC_PLAIN, cnt, G);
            float amp = 0.f;
            const int rs = solve_moments_refined<DIM, DEG, MODE_MAP, float>(acc, nullptr, bound, yh, yl,
                                                                            nullptr, &amp);
            if (rs == 1 && amp <= bound) {
                rows64 = amp > (float)AMP_SHAPE;
                if (rows64) {
#pragma unroll
                    for (int k = 0; k < M; k++) y64[k] = (double)yh[k] + (double)yl[k];
                }
            } else if (rs == 0) {
                double m64[NM], a64 = 0.0;
#pragma unroll
                for (int i = 0; i < NM; i++) m64[i] = (double)acc[i];
                if (solve_moments<DIM, DEG, MODE_MAP>(m64, 0.0, TAU32, y64, nullptr, &a64) &&
                    (float)a64 <= bound) {
                    rows64 = true;
                } else {
                    fp64 = true;
                }
            } else {
                fp64 = true;
            }
        }
        if (fp64) {   // the FP64 assembly and solve
            double m64[NM];
#pragma unroll
            for (int i = 0; i < NM; i++) m64[i] = 0.0;
            const double inv_r = R.inv_r;
            auto moments64 = [&](int n) {
                for (int e0 = 0; e0 < n; e0 += G) {
                    const int e = e0 + gl;
                    if (e < n) {
                        const int j = stg[e];
                        double dx[3] = {0.0, 0.0, 0.0};
#pragma unroll
                        for (int d = 0; d < DIM; d++) dx[d] = __dsub_rn(R.x64[d * R.ns + j], tx[d]);
                        accumulate<DIM, DEG, MODE_MAP, double, NM>(m64, dx, 0.0, R.weight, inv_r, nullptr);
                    }
                }
            };
            if (have_all) {
                moments64(staged);
            } else {
                walk_select<DIM, G>(R, g, ct, fr, thi, tlo, tx, rA, rE, stg, STG, gl, gmask, staged,
                                    spilled, moments64);
                moments64(staged);
            }
#pragma unroll
            for (int i = 0; i < NM; i++) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) m64[i] += __shfl_xor_sync(gmask, m64[i], o);
            }
            double a64 = 0.0, rho = 1.0;
            if (!solve_moments<DIM, DEG, MODE_MAP>(m64, 0.0, TAU64, y64, nullptr, &a64, nullptr, &rho))
                st = PCMS_TARGET_ILL_CONDITIONED;
            rows64 = true;
            // The status is decided in the target-centred basis (the definition's). FP64
            // normal equations still lose digits with amp (c_0 to about 15 amp 2^-53, more
            // for fits through about m points), so a target with amp > AMP_FP64 is assembled
            // and solved once more in the re-centred basis of its neighbours (centroid c and
            // spread s from these moments), where the value is the fitted polynomial at
            // u'_t = -c/s; if that solve passes its guard, it replaces the first.
            if (DEG >= 1 && st == PCMS_TARGET_OK && a64 > AMP_FP64) {
                const float4 b = recentre_basis<DIM>(m64);
                if (!is_target_centred(b)) {
                    const double bd[4] = {(double)b.x, (double)b.y, (double)b.z, (double)b.w};
#pragma unroll
                    for (int i = 0; i < NM; i++) m64[i] = 0.0;
                    auto moments64b = [&](int n) {
                        for (int e0 = 0; e0 < n; e0 += G) {
                            const int e = e0 + gl;
                            if (e < n) {
                                const int j = stg[e];
                                double dx[3] = {0.0, 0.0, 0.0};
#pragma unroll
                                for (int d = 0; d < DIM; d++) dx[d] = __dsub_rn(R.x64[d * R.ns + j], tx[d]);
                                accumulate<DIM, DEG, MODE_MAP, double, NM>(m64, dx, 0.0, R.weight, inv_r, bd);
                            }
                        }
                    };
                    if (have_all) {
                        moments64b(staged);
                    } else {
                        walk_select<DIM, G>(R, g, ct, fr, thi, tlo, tx, rA, rE, stg, STG, gl, gmask,
                                            staged, spilled, moments64b);
                        moments64b(staged);
                    }
#pragma unroll
                    for (int i = 0; i < NM; i++) {
#pragma unroll
                        for (int o = G / 2; o > 0; o >>= 1) m64[i] += __shfl_xor_sync(gmask, m64[i], o);
                    }
                    double at[M], y2[M], a2 = 0.0;
                    basis_at_target<DIM, DEG>(b, at);
                    double rho2 = 1.0;
                    if (solve_moments<DIM, DEG, MODE_MAP>(m64, 0.0, TAU64, y2, nullptr, &a2, at, &rho2)) {
#pragma unroll
                        for (int k = 0; k < M; k++) y64[k] = y2[k];
                        rbasis = b;
                        recentred = true;
                        a64 = a2;
                        rho = rho2;
                    }
                }
            }
            if (DEG >= 1 && st == PCMS_TARGET_OK && a64 > AMP_QR * rho && cnt <= QR_MAX && gl == 0) {
                const unsigned q = atomicAdd(&hdr->n_qr, 1u);
                if (q < hdr->qr_cap) hdr->qr_list[q] = make_int2(r, (int)t);
            }
        }

        // operator rows applied to the fields: out_f = sum_j w_j a(u_j)^T y fs[j][f].
        // FP32 rows (amp <= AMP_SHAPE, so sum_j |N_j| <= amp is small) accumulate in FP32;
        // FP64 rows accumulate in FP64: their |N_j| can be large with cancelling signs
        // (extrapolating targets with about m neighbours), and FP32 sums of such terms lose
        // the bound.
        if (st == PCMS_TARGET_OK) {
            if (rows64) {
                double o[16];
#pragma unroll
                for (int f = 0; f < 16; f++) o[f] = 0.0;
                auto rows = [&](int n) {
                    for (int e0 = 0; e0 < n; e0 += G) {
                        const int e = e0 + gl;
                        if (e >= n) continue;
                        const int j = stg[e];
                        double dx[3] = {0.0, 0.0, 0.0};
#pragma unroll
                        for (int d = 0; d < DIM; d++) dx[d] = __dsub_rn(R.x64[d * R.ns + j], tx[d]);
                        double d2 = dx[0] * dx[0] + dx[1] * dx[1];
                        if (DIM == 3) d2 += dx[2] * dx[2];
                        const double w = weight_value<double>(R.weight, sqrt(d2) * R.inv_r);
                        double u[3];
                        const double bd[4] = {(double)rbasis.x, (double)rbasis.y, (double)rbasis.z,
                                              (double)rbasis.w};
                        basis_offsets<DIM, double>(dx, R.inv_r, recentred ? bd : nullptr, u);
                        double a[M];
                        a[0] = 1.0;
                        double dot = y64[0];
                        sfor<M - 1>([&](auto I) {
                            constexpr int p = decltype(I)::value + 1;
                            a[p] = a[mono_parent(DIM, p)] * u[mono_var(DIM, p)];
                            dot += a[p] * y64[p];
                        });
                        apply_row<double>(R, j, w * dot, o);
                    }
                };
                if (have_all) {
                    rows(staged);
                } else {
                    walk_select<DIM, G>(R, g, ct, fr, thi, tlo, tx, rA, rE, stg, STG, gl, gmask,
                                        staged, spilled, rows);
                    rows(staged);
                }
                finish_rows<G>(R, o, t, gl, gmask);
            } else {
                float o[16];
#pragma unroll
                for (int f = 0; f < 16; f++) o[f] = 0.f;
                auto rows = [&](int n) {
                    for (int e0 = 0; e0 < n; e0 += G) {
                        const int e = e0 + gl;
                        if (e >= n) continue;
                        const int j = stg[e];
                        float dx[3];
                        offsets32<DIM>(R, j, thi, tlo, dx);
                        float d2 = dx[0] * dx[0] + dx[1] * dx[1];
                        if (DIM == 3) d2 += dx[2] * dx[2];
                        const float w = weight_value<float>(R.weight, sqrt_approx(d2) * R.inv_rf);
                        float u[3];
                        basis_offsets<DIM, float>(dx, R.inv_rf, nullptr, u);
                        float a[M];
                        a[0] = 1.f;
                        float dot = yh[0];
                        sfor<M - 1>([&](auto I) {
                            constexpr int p = decltype(I)::value + 1;
                            a[p] = a[mono_parent(DIM, p)] * u[mono_var(DIM, p)];
                            dot += a[p] * yh[p];
                        });
                        apply_row<float>(R, j, w * dot, o);
                    }
                };
                if (have_all) {
                    rows(staged);
                } else {
                    walk_select<DIM, G>(R, g, ct, fr, thi, tlo, tx, rA, rE, stg, STG, gl, gmask,
                                        staged, spilled, rows);
                    rows(staged);
                }
                finish_rows<G>(R, o, t, gl, gmask);
            }
        } else {
            const float nan = __int_as_float(0x7fc00000);
            for (int f = gl; f < R.nf; f += G) R.out[(int64_t)f * R.nt + t] = nan;
        }
        if (gl == 0 && R.status) R.status[t] = (int8_t)st;
        __syncwarp(gmask);   // the stage is reused by the group's next target
    }
}

// ------------------------------------------------------------------------------------
// k_batch_qr: the listed targets by Householder QR (one warp per target)
// ------------------------------------------------------------------------------------
// For target t of problem r: the selected sources again (the same walk and decision as
// k_batch_mls), B = diag(sqrt(w)) A with A the target-centred, radius-scaled monomials,
// Householder QR of B with the definition's rank test (|R_kk| <= 1e-7 of column k's norm:
// ill-conditioned), then the operator row N = diag(sqrt(w)) Q R^-T e_1 and out_f = sum_i
// N_i f_i, all in FP64; the values (and the status) replace the normal equations' ones.
template <int DIM, int DEG>
__global__ void __launch_bounds__(QR_WARPS * 32) k_batch_qr(BatchHeader* hdr, const BatchReq* reqs) {
    constexpr int M = mono_count(DIM, DEG);
    __shared__ QrSpace<M> ws[QR_WARPS];
    __shared__ int32_t jl[QR_WARPS][QR_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned nq = min(hdr->n_qr, hdr->qr_cap);
    for (unsigned e = blockIdx.x * QR_WARPS + w; e < nq; e += gridDim.x * QR_WARPS) {
        const int2 rt = hdr->qr_list[e];
        const BatchReq& R = reqs[rt.x];
        const int64_t t = rt.y;
        Grid g;
        g.dim = DIM;
        g.n[0] = R.n[0];
        g.n[1] = R.n[1];
        g.n[2] = R.n[2];
        g.ncell = (int64_t)R.n[0] * R.n[1] * R.n[2];
        g.lo[0] = R.lo[0];
        g.lo[1] = R.lo[1];
        g.lo[2] = R.lo[2];
        g.h = R.h;
        g.inv_h = R.inv_h;
        double tx[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < DIM; d++) tx[d] = R.tgt[d * R.nt + t];
        const int cnt = qr_collect<DIM>(g, R.cell_start, R.x64, R.ns, tx, R.radius, R.r2, R.weight,
                                        jl[w], QR_MAX, lane);
        if (cnt < M) continue;   // over the cap: keep the normal equations' values
        double n0, n1;
        const bool ok = qr_row<DIM, DEG>(R.x64, R.ns, jl[w], cnt, tx, R.radius, R.weight, ws[w],
                                         lane, n0, n1);
        if (!ok) {
            const float nan = __int_as_float(0x7fc00000);
            for (int f = lane; f < R.nf; f += 32) R.out[(int64_t)f * R.nt + t] = nan;
            if (lane == 0 && R.status) R.status[t] = PCMS_TARGET_ILL_CONDITIONED;
            __syncwarp();
            continue;
        }
        const int j0 = lane < cnt ? jl[w][lane] : 0;
        const int j1 = lane + 32 < cnt ? jl[w][lane + 32] : 0;
        for (int f = 0; f < R.nf; f++) {
            double v = 0.0;
            if (lane < cnt) v += n0 * (double)R.fs[(int64_t)j0 * R.fp + f];
            if (lane + 32 < cnt) v += n1 * (double)R.fs[(int64_t)j1 * R.fp + f];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) R.out[(int64_t)f * R.nt + t] = (float)v;
        }
        __syncwarp();
    }
}

template <int DIM, int DEG, int G>
void launch_mls_t(int per_sm, BatchHeader* hdr, const BatchReq* reqs, cudaStream_t s) {
    k_batch_mls<DIM, DEG, G><<<num_sms() * per_sm, MLS_THREADS, 0, s>>>(hdr, reqs);
}

template <int DIM, int DEG, int G>
int occupancy_t() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_mls<DIM, DEG, G>,
                                                      MLS_THREADS, 0) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    return per_sm;
}

// class index: (dim - 2) * 6 + degree * 2 + (G == 32)
// the class's two kernels on s; traced = false while a graph is being captured (the
// graph's launches are counted when it is launched)
template <int DIM, int DEG, int G>
void launch_class_t(BatchHeader* hdr, BatchReq* reqs, cudaStream_t s, bool traced) {
    static const int per_sm = occupancy_t<DIM, DEG, G>();
    {
        TraceScope ts(traced ? "batch_sort" : nullptr, s);
        k_batch_sort<DIM><<<num_sms(), SORT_THREADS, 0, s>>>(hdr, reqs);
    }
    PCMS_LAUNCH_CHECK("k_batch_sort");
    {
        TraceScope ts(traced ? "batch_mls" : nullptr, s);
        launch_mls_t<DIM, DEG, G>(per_sm, hdr, reqs, s);
    }
    PCMS_LAUNCH_CHECK("k_batch_mls");
    if (DEG >= 1) {
        static const int qr_per_sm = [] {
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_qr<DIM, DEG>, QR_WARPS * 32, 0) !=
                    cudaSuccess || n < 1) {
                (void)cudaGetLastError();
                n = 1;
            }
            return n;
        }();
        TraceScope ts(traced ? "batch_qr" : nullptr, s);
        k_batch_qr<DIM, DEG><<<num_sms() * qr_per_sm, QR_WARPS * 32, 0, s>>>(hdr, reqs);
    }
    PCMS_LAUNCH_CHECK("k_batch_qr");
}

void launch_class(int ci, BatchHeader* hdr, BatchReq* reqs, cudaStream_t s, bool traced) {
    switch (ci) {
    case 0: return launch_class_t<2, 0, 8>(hdr, reqs, s, traced);
    case 1: return launch_class_t<2, 0, 32>(hdr, reqs, s, traced);
    case 2: return launch_class_t<2, 1, 8>(hdr, reqs, s, traced);
    case 3: return launch_class_t<2, 1, 32>(hdr, reqs, s, traced);
    case 4: return launch_class_t<2, 2, 8>(hdr, reqs, s, traced);
    case 5: return launch_class_t<2, 2, 32>(hdr, reqs, s, traced);
    case 6: return launch_class_t<3, 0, 8>(hdr, reqs, s, traced);
    case 7: return launch_class_t<3, 0, 32>(hdr, reqs, s, traced);
    case 8: return launch_class_t<3, 1, 8>(hdr, reqs, s, traced);
    case 9: return launch_class_t<3, 1, 32>(hdr, reqs, s, traced);
    case 10: return launch_class_t<3, 2, 8>(hdr, reqs, s, traced);
    case 11: return launch_class_t<3, 2, 32>(hdr, reqs, s, traced);
    default: fail(PCMS_ERR_INVALID_ARG, "internal: batch class");
    }
}

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

int field_pad(int nf) { return nf == 1 ? 1 : (nf + 3) / 4 * 4; }

int64_t cell_budget(int64_t ns) { return std::min<int64_t>(4 * ns + 64, int64_t(1) << 24); }

// Expected neighbours per target: sources per unit volume of their box, taken as the unit
// box, times the ball's volume; 32 lanes per target from 160 on (as the general path).
int lanes_for(const pcms_batch_item& it) {
    const double r = it.radius;
    const double ball = it.dim == 2 ? M_PI * r * r : 4.0 / 3.0 * M_PI * r * r * r;
    return (double)it.n_src * ball >= 160.0 ? 32 : 8;
}

}  // namespace

int batch_class_of(const pcms_batch_item& it) {
    return (it.dim - 2) * 6 + it.basis_degree * 2 + (lanes_for(it) == 32 ? 1 : 0);
}

int64_t batch_item_bytes(const pcms_batch_item& it) {
    const int64_t ns = it.n_src, cap = cell_budget(ns);
    int64_t b = align256(4 * (cap + 1)) + align256(4 * cap) + 2 * align256(4 * ns) +
                align256(8 * it.dim * ns) + align256(16 * ns) + (it.dim == 3 ? align256(8 * ns) : 0) +
                align256(4 * (int64_t)field_pad(it.n_fields) * ns);
    return b;
}

std::string batch_check_item(const pcms_batch_item& it) {
    if (it.dim != 2 && it.dim != 3) return "dim must be 2 or 3";
    if (it.basis_degree < 0 || it.basis_degree > 2) return "basis_degree must be 0, 1 or 2";
    if (!std::isfinite(it.radius) || !(it.radius > 0.0)) return "radius must be finite and > 0";
    if ((int)it.weight < 0 || (int)it.weight > 8) return "bad weight kind";
    if (it.n_src < 0 || it.n_tgt < 0) return "negative point count";
    if (it.n_src > PCMS_BATCH_MAX_POINTS || it.n_tgt > PCMS_BATCH_MAX_POINTS)
        return "n_src and n_tgt must be at most PCMS_BATCH_MAX_POINTS";
    if (it.n_fields < 1 || it.n_fields > 16) return "n_fields must be in 1..16";
    if (it.n_src > 0 && (!it.src_pts || !it.fields)) return "src_pts or fields is NULL";
    if (it.n_tgt > 0 && (!it.tgt_pts || !it.out)) return "tgt_pts or out is NULL";
    return "";
}

BatchExec::BatchExec(bool use_graphs) : graphs_(use_graphs) {
    const size_t per_class = sizeof(BatchHeader) + sizeof(BatchReq) * PCMS_BATCH_MAX_ITEMS;
    PCMS_CU(cudaMalloc(&table_d_, per_class * BATCH_CLASSES));
    if (graphs_) {
        PCMS_CU(cudaHostAlloc(&table_h_, per_class * BATCH_CLASSES, cudaHostAllocDefault));
        PCMS_CU(cudaHostAlloc(&err_h_, sizeof(int32_t) * PCMS_BATCH_MAX_ITEMS * BATCH_CLASSES,
                              cudaHostAllocDefault));
    } else {
        table_v_.resize(per_class * BATCH_CLASSES);
        err_v_.resize((size_t)PCMS_BATCH_MAX_ITEMS * BATCH_CLASSES);
        table_h_ = table_v_.data();
        err_h_ = err_v_.data();
    }
    std::memset(table_h_, 0, per_class * BATCH_CLASSES);
}

// Captures, once, the class's table copy and kernels on s into a graph. Captures are
// serialised across the process; any failure leaves the class on direct launches.
void BatchExec::capture(int c, void* td, const void* th, size_t bytes, BatchHeader* hdr_d,
                        BatchReq* req_d, cudaStream_t s) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaMemcpyAsync(td, th, bytes, cudaMemcpyHostToDevice, s);
        if (le == cudaSuccess) {
            try {
                launch_class(c, hdr_d, req_d, s, false);
            } catch (const PcmsError&) {
                le = cudaErrorUnknown;
            }
        }
        e = cudaStreamEndCapture(s, &gr);   // ends the capture whatever happened inside it
        if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess && gr) e = cudaGraphInstantiate(&ex, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess || !ex) {
        (void)cudaGetLastError();
        no_graph_[c] = true;
        exec_[c] = nullptr;
        return;
    }
    exec_[c] = ex;
}

BatchExec::~BatchExec() {
    for (auto& e : exec_)
        if (e) cudaGraphExecDestroy(e);
    if (table_d_) cudaFree(table_d_);
    if (graphs_) {
        if (table_h_) cudaFreeHost(table_h_);
        if (err_h_) cudaFreeHost(err_h_);
    }
}

void BatchExec::run(const pcms_batch_item* items, int n, int32_t* result, cudaStream_t s) {
    if (n <= 0) return;
    if (graphs_ && !result) fail(PCMS_ERR_INVALID_ARG, "internal: a graph batch needs its results read");
    if (n > PCMS_BATCH_MAX_ITEMS) fail(PCMS_ERR_INVALID_ARG, "more than PCMS_BATCH_MAX_ITEMS items");
    for (int i = 0; i < n; i++) {
        const std::string e = batch_check_item(items[i]);
        if (!e.empty()) fail(PCMS_ERR_INVALID_ARG, "item " + std::to_string(i) + ": " + e);
    }
    std::vector<int> cls(n);
    int64_t arena = 0;
    for (int i = 0; i < n; i++) {
        cls[i] = batch_class_of(items[i]);
        arena += batch_item_bytes(items[i]) + align256(8 * std::max<int64_t>(items[i].n_tgt, 1));
    }
    DBuf mem(std::max<int64_t>(arena, 256), s);
    char* base = (char*)mem.p;
    const size_t per_class = sizeof(BatchHeader) + sizeof(BatchReq) * PCMS_BATCH_MAX_ITEMS;
    std::vector<std::vector<int>> members(BATCH_CLASSES);
    for (int i = 0; i < n; i++) members[cls[i]].push_back(i);
    bool any = false;
    for (int c = 0; c < BATCH_CLASSES; c++) {
        if (members[c].empty()) continue;
        const int G = (c & 1) ? 32 : 8;
        const int tile = (MLS_THREADS / 32) * (32 / G);
        char* th = (char*)table_h_ + per_class * c;
        char* td = (char*)table_d_ + per_class * c;
        auto* hh = reinterpret_cast<BatchHeader*>(th);
        auto* rh = reinterpret_cast<BatchReq*>(th + sizeof(BatchHeader));
        std::memset(th, 0, per_class);
        long long tiles = 0;
        int k = 0;
        for (int i : members[c]) {
            const pcms_batch_item& it = items[i];
            BatchReq& q = rh[k++];
            const int64_t ns = it.n_src, cap = cell_budget(ns);
            q.src = it.src_pts;
            q.tgt = it.tgt_pts;
            q.fields = it.fields;
            q.out = it.out;
            q.status = it.target_status;
            q.ns = ns;
            q.nt = it.n_tgt;
            q.cap_cells = cap;
            q.tile0 = tiles;
            tiles += (it.n_tgt + tile - 1) / tile;
            q.nf = it.n_fields;
            q.fp = field_pad(it.n_fields);
            q.weight = (int)it.weight;
            q.radius = it.radius;
            q.r2 = it.radius * it.radius;
            q.inv_r = 1.0 / it.radius;
            q.r2f = (float)(it.radius * it.radius);
            q.inv_rf = (float)(1.0 / it.radius);
            auto take = [&](int64_t bytes) {
                char* p = base;
                base += align256(bytes);
                return p;
            };
            q.cell_start = (int32_t*)take(4 * (cap + 1));
            q.cursor = (int32_t*)take(4 * cap);
            q.keys = (int32_t*)take(4 * ns);
            q.perm = (int32_t*)take(4 * ns);
            q.x64 = (double*)take(8 * it.dim * ns);
            q.hl0 = (float4*)take(16 * ns);
            q.hl1 = it.dim == 3 ? (float2*)take(8 * ns) : nullptr;
            q.fs = (float*)take(4 * (int64_t)q.fp * ns);
        }
        hh->n_req = k;
        hh->total_tiles = tiles;
        hh->next = 0;
        int64_t class_targets = 0;
        for (int i : members[c]) class_targets += items[i].n_tgt;
        hh->qr_cap = (unsigned)std::max<int64_t>(class_targets, 1);
        hh->qr_list = (int2*)base;
        base += align256(8 * (int64_t)hh->qr_cap);
        hh->n_qr = 0;
        if (tiles == 0 && k == 0) continue;
        any = true;
        const size_t bytes = sizeof(BatchHeader) + sizeof(BatchReq) * k;
        auto* hdr_d = reinterpret_cast<BatchHeader*>(td);
        auto* req_d = reinterpret_cast<BatchReq*>(td + sizeof(BatchHeader));
        if (graphs_ && !trace_timing() && !no_graph_[c]) {
            // one graph per class: the table copy and the kernels, with fixed arguments (the
            // table region of the class); the table carries every per-batch value
            if (!exec_[c]) capture(c, td, th, per_class, hdr_d, req_d, s);
        }
        if (exec_[c]) {
            if (trace_on()) {   // count mode: the graph's kernels
                PCMS_TRACE("batch_sort", s);
                PCMS_TRACE("batch_mls", s);
                if (c / 2 % 3 != 0) PCMS_TRACE("batch_qr", s);
            }
            PCMS_CU(cudaGraphLaunch(exec_[c], s));
        } else {
            PCMS_CU(cudaMemcpyAsync(td, th, bytes, cudaMemcpyHostToDevice, s));
            launch_class(c, hdr_d, req_d, s, true);
        }
    }
    if (!any || !result) return;
    for (int c = 0; c < BATCH_CLASSES; c++) {
        if (members[c].empty()) continue;
        const auto* hdr_d = reinterpret_cast<const BatchHeader*>((char*)table_d_ + per_class * c);
        PCMS_CU(cudaMemcpyAsync(err_h_ + PCMS_BATCH_MAX_ITEMS * c, hdr_d->err,
                                sizeof(int32_t) * members[c].size(), cudaMemcpyDeviceToHost, s));
    }
    PCMS_CU(cudaStreamSynchronize(s));
    for (int c = 0; c < BATCH_CLASSES; c++) {
        int k = 0;
        for (int i : members[c]) {
            const int e = err_h_[PCMS_BATCH_MAX_ITEMS * c + k++];
            result[i] = e ? PCMS_ERR_INVALID_ARG : PCMS_OK;
        }
    }
}

}  // namespace pcms
