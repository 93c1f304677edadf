// apply.cu -- evaluation of a cached MLS operator on one or many fields (out = N f, the
// transferred values of Sec. 3.2.1), and export of the operator in the caller's orders.
//
// Data flow of one apply (all HBM-streaming kernels):
//   1. k_fields_to_sorted: fields [F][ns] (caller order) -> fs [ns][FP] (sorted by cell,
//      fields interleaved, FP = F rounded up to the vector width). Reads are coalesced over
//      the caller index; each source writes one contiguous FP-element row.
//   2. k_spmm: one warp per target row (targets sorted by cell), lanes split into
//      32/NV nnz slots x NV vectors of fields; each slot reads (col, val) once and NV
//      vectors of the source's field row. Blocks take chunks of consecutive rows, so
//      neighbouring targets, which share most sources, are in flight together and the
//      gathered field rows are served mostly from L1/L2.
//   3. k_stage_to_caller: out[f][i] = stage[inv_t[i]][f], coalesced writes per field.
#include <algorithm>

#include "pcms_internal.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

int blocks_for(int64_t n, int threads, int per_sm = 32) {
    int64_t need = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * per_sm));
}

// Rows are handed out in chunks of SPMM_ROWS consecutive targets (an atomic counter), so a
// block's warps work on neighbouring targets at the same time and share their gathered field
// rows in L1; chunks also balance rows of uneven length (the denser slab of the 3D case).
constexpr int SPMM_ROWS = 128;

// persistent grid of the apply: as many 256-thread blocks as fit on the GPU at once (they
// take chunks of rows from a counter), at most one per chunk
template <typename K>
int spmm_blocks(K kernel, int64_t nt) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    const int64_t chunks = (nt + SPMM_ROWS - 1) / SPMM_ROWS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)num_sms() * per_sm));
}

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

// caller-order fields -> sorted, interleaved rows; fp is 1 or a multiple of the vector width,
// each row is written with vector stores
template <typename T>
__global__ void k_fields_to_sorted(const T* __restrict__ f, int nf, int fp, int64_t ns,
                                   const int32_t* __restrict__ inv, T* __restrict__ fs) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        T* row = fs + (int64_t)inv[i] * fp;
        if (fp == 1) {
            row[0] = f[i];
            continue;
        }
        for (int v = 0; v < fp / W; v++) {
            T tmp[W];
#pragma unroll
            for (int c = 0; c < W; c++) {
                const int k = v * W + c;
                tmp[c] = k < nf ? f[(int64_t)k * ns + i] : T(0);
            }
            V x;
            memcpy(&x, tmp, sizeof(V));
            reinterpret_cast<V*>(row)[v] = x;
        }
    }
}

template <typename V, typename T>
__device__ __forceinline__ void fma_vec(V& acc, T a, const V& x);
template <>
__device__ __forceinline__ void fma_vec<float4, float>(float4& acc, float a, const float4& x) {
    acc.x = fmaf(a, x.x, acc.x); acc.y = fmaf(a, x.y, acc.y);
    acc.z = fmaf(a, x.z, acc.z); acc.w = fmaf(a, x.w, acc.w);
}
template <>
__device__ __forceinline__ void fma_vec<double2, double>(double2& acc, double a, const double2& x) {
    acc.x = fma(a, x.x, acc.x); acc.y = fma(a, x.y, acc.y);
}
// Sum over the slots of a row's partial vectors (lane = slot * NV + vi), with the vector's
// components spread over the lanes instead of reduced whole: the first exchange (lanes 16
// apart) halves the components a lane keeps, the second (8 apart, float4 only) halves them
// again, the rest are plain. On return the lane holds the total of component *comp of vector
// vi; the lanes that hold distinct totals are those with (lane & writer_mask) == 0.
template <int NV>
__device__ __forceinline__ float slot_total(const float4& a, int lane, int* comp) {
    static_assert(NV <= 8, "lanes 8 and 16 apart must hold different slots");
    const bool h = lane & 16, q = lane & 8;
    const float k0 = (h ? a.z : a.x) + __shfl_xor_sync(0xffffffffu, h ? a.x : a.z, 16);
    const float k1 = (h ? a.w : a.y) + __shfl_xor_sync(0xffffffffu, h ? a.y : a.w, 16);
    float k = (q ? k1 : k0) + __shfl_xor_sync(0xffffffffu, q ? k0 : k1, 8);
#pragma unroll
    for (int o = NV; o < 8; o <<= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    *comp = (h ? 2 : 0) + (q ? 1 : 0);
    return k;
}
template <int NV>
__device__ __forceinline__ double slot_total(const double2& a, int lane, int* comp) {
    const bool h = lane & 16;
    double k = (h ? a.y : a.x) + __shfl_xor_sync(0xffffffffu, h ? a.x : a.y, 16);
#pragma unroll
    for (int o = NV; o < 16; o <<= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    *comp = h ? 1 : 0;
    return k;
}
template <typename T, int NV>
constexpr int writer_mask() {
    return sizeof(T) == 4 ? 8 - NV : 16 - NV;
}

template <typename T>
__device__ __forceinline__ T quiet_nan();
template <>
__device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ double quiet_nan<double>() {
    return __longlong_as_double(0x7ff8000000000000LL);
}

__device__ __forceinline__ int64_t spmm_next_chunk(unsigned long long* next) {
    __shared__ long long chunk_s;
    __syncthreads();   // the previous chunk's start has been read by every thread
    if (threadIdx.x == 0) chunk_s = (long long)atomicAdd(next, (unsigned long long)SPMM_ROWS);
    __syncthreads();
    return chunk_s;
}

// One warp per target row; lanes = 32/NV slots x NV vectors of W fields (fp = NV*W).
// Nonzeros are taken 32 at a time: each lane loads one (col, val) pair with a coalesced load,
// the columns are redistributed by shuffles, and every lane then has NV independent
// field-row gathers in flight. A row's first 64 (col, val) pairs are loaded together, and the
// next row's offsets and first 32 pairs while the current row is gathered. Rows whose target
// status is not OK produce NaN.
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_spmm_vec(int64_t nt, const int64_t* __restrict__ off,
                                                  const int32_t* __restrict__ cnt,
                                                  const int32_t* __restrict__ cols,
                                                  const T* __restrict__ vals,
                                                  const T* __restrict__ fs,
                                                  const int8_t* __restrict__ status,
                                                  T* __restrict__ stage,
                                                  unsigned long long* next) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    constexpr int SLOTS = 32 / NV;
    const int lane = threadIdx.x & 31;
    const int slot = lane / NV, vi = lane % NV;
    const int nwb = blockDim.x >> 5, wib = threadIdx.x >> 5;
    for (;;) {
        const int64_t c0 = spmm_next_chunk(next);
        if (c0 >= nt) break;
        const int64_t c1 = min(c0 + (int64_t)SPMM_ROWS, nt);
        int64_t t = c0 + wib;
        int64_t a = 0, b = 0;
        int32_t jA = 0;
        T wA = T(0);
        if (t < c1) {
            a = off[t];
            b = a + cnt[t];
            if (a + lane < b) {
                jA = __ldg(cols + a + lane);
                wA = __ldg(vals + a + lane);
            }
        }
        for (; t < c1; t += nwb) {
            // the row's second 32 pairs, and the next row's offsets
            int32_t jB = 0;
            T wB = T(0);
            if (a + 32 + lane < b) {
                jB = __ldg(cols + a + 32 + lane);
                wB = __ldg(vals + a + 32 + lane);
            }
            const int64_t tn = t + nwb;
            int64_t an = 0, bn = 0;
            if (tn < c1) {
                an = off[tn];
                bn = an + cnt[tn];
            }
            V acc{};
            for (int64_t e0 = a; e0 < b; e0 += 32) {
                if (e0 >= a + 64) {   // rows longer than 64 nonzeros
                    jB = e0 + lane < b ? __ldg(cols + e0 + lane) : 0;
                    wB = e0 + lane < b ? __ldg(vals + e0 + lane) : T(0);
                }
                const bool first = e0 == a;
                const int32_t jl = first ? jA : jB;
                const T wl = first ? wA : wB;
                V x[NV];
#pragma unroll
                for (int s = 0; s < NV; s++) {
                    const int k = s * SLOTS + slot;
                    const int32_t j = __shfl_sync(0xffffffffu, jl, k);
                    x[s] = e0 + k < b ? *reinterpret_cast<const V*>(fs + (int64_t)j * (NV * W) + vi * W)
                                      : V{};
                }
#pragma unroll
                for (int s = 0; s < NV; s++)
                    fma_vec<V, T>(acc, __shfl_sync(0xffffffffu, wl, s * SLOTS + slot), x[s]);
            }
            jA = 0;
            wA = T(0);
            if (an + lane < bn) {   // the next row's first 32 pairs
                jA = __ldg(cols + an + lane);
                wA = __ldg(vals + an + lane);
            }
            int comp;
            const T tot = slot_total<NV>(acc, lane, &comp);
            if ((lane & writer_mask<T, NV>()) == 0)
                stage[t * (NV * W) + vi * W + comp] =
                    status[t] == PCMS_TARGET_OK ? tot : quiet_nan<T>();
            a = an;
            b = bn;
        }
    }
}

// FP32 fields, fp = 4 NV (NV = 1, 2, 4 float4 vectors per source row): NV lanes per nonzero,
// each lane one float4 of the row, 32 / NV nonzeros per warp step. The lanes of a nonzero
// load its (col, val) together (one broadcast transaction), so no shuffles redistribute
// them; steps are unrolled four times, so four field-row gathers per lane are in flight.
// 32 registers: eight blocks (64 warps) per SM. (Loading the next row's (col, val) pairs
// behind the current row's gathers took 48 registers and measured slower: 3.0 against 2.5
// ms on the 8M 3D operator with 16 fields. So did staging each row's pairs in shared memory
// by cp.async two rows ahead, the row offsets a row before that: 40 registers, 48 warps per
// SM, 3.3 ms. The field-row gathers and the warps in flight decide the time, not the chain
// of loads that leads to them. Handing each SM its own contiguous range of row chunks, so
// that its blocks share neighbouring sources in L1, measured 3.1 ms.)
// At the row's end the lanes holding the same vector position are summed (xor shuffles
// over the 32 / NV nonzero slots) and lanes 0 .. NV-1 store the row. One warp per row,
// rows in chunks from the counter as k_spmm_vec.
template <int NV>
__global__ void __launch_bounds__(256) k_spmm_q(int64_t nt, const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ cnt,
                                                const int32_t* __restrict__ cols,
                                                const float* __restrict__ vals,
                                                const float* __restrict__ fs,
                                                const int8_t* __restrict__ status,
                                                float* __restrict__ stage,
                                                unsigned long long* next) {
    constexpr int SL = 32 / NV;   // nonzero slots per step
    const int lane = threadIdx.x & 31;
    const int slot = lane / NV, vi = lane % NV;
    const int nwb = blockDim.x >> 5, wib = threadIdx.x >> 5;
    const float4* __restrict__ f4 = reinterpret_cast<const float4*>(fs);
    for (;;) {
        const int64_t c0 = spmm_next_chunk(next);
        if (c0 >= nt) break;
        const int64_t c1 = min(c0 + (int64_t)SPMM_ROWS, nt);
        for (int64_t t = c0 + wib; t < c1; t += nwb) {
            const int64_t a = off[t], b = a + cnt[t];
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            int64_t e = a + slot;
            for (; e + 3 * SL < b; e += 4 * SL) {
                int32_t j[4];
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    j[u] = __ldg(cols + e + u * SL);
                    w[u] = __ldg(vals + e + u * SL);
                }
                float4 x[4];
#pragma unroll
                for (int u = 0; u < 4; u++) x[u] = __ldg(f4 + (int64_t)j[u] * NV + vi);
#pragma unroll
                for (int u = 0; u < 4; u++) fma_vec<float4, float>(acc, w[u], x[u]);
            }
            for (; e < b; e += SL) {
                const int32_t j = __ldg(cols + e);
                const float w = __ldg(vals + e);
                fma_vec<float4, float>(acc, w, __ldg(f4 + (int64_t)j * NV + vi));
            }
#pragma unroll
            for (int o = NV; o < 32; o <<= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
                acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
            }
            if (lane < NV) {
                const float nan = quiet_nan<float>();
                reinterpret_cast<float4*>(stage)[t * NV + vi] =
                    status[t] == PCMS_TARGET_OK ? acc : make_float4(nan, nan, nan, nan);
            }
        }
    }
}

// one field: lanes over nonzeros, 64 in flight, rows in chunks as above
template <typename T>
__global__ void __launch_bounds__(256) k_spmm_1(int64_t nt, const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ cnt,
                                                const int32_t* __restrict__ cols,
                                                const T* __restrict__ vals,
                                                const T* __restrict__ fs,
                                                const int8_t* __restrict__ status,
                                                T* __restrict__ stage,
                                                unsigned long long* next) {
    const int lane = threadIdx.x & 31;
    const int nwb = blockDim.x >> 5, wib = threadIdx.x >> 5;
    for (;;) {
        const int64_t c0 = spmm_next_chunk(next);
        if (c0 >= nt) break;
        const int64_t c1 = min(c0 + (int64_t)SPMM_ROWS, nt);
        for (int64_t t = c0 + wib; t < c1; t += nwb) {
            const int64_t a = off[t], b = a + cnt[t];
            T acc = T(0);
            for (int64_t e = a + lane; e < b; e += 64) {
                const bool two = e + 32 < b;
                const int32_t j0 = __ldg(cols + e);
                const int32_t j1 = two ? __ldg(cols + e + 32) : 0;
                const T w0 = __ldg(vals + e);
                const T w1 = two ? __ldg(vals + e + 32) : T(0);
                const T x0 = fs[j0];
                const T x1 = two ? fs[j1] : T(0);
                acc += w0 * x0;
                acc += w1 * x1;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) stage[t] = status[t] == PCMS_TARGET_OK ? acc : quiet_nan<T>();
        }
    }
}

template <typename T>
__global__ void k_stage_to_caller(const T* __restrict__ stage, int fp, int nf, int64_t nt,
                                  const int32_t* __restrict__ inv_t, T* __restrict__ out) {
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const T* row = stage + (int64_t)inv_t[i] * fp;
        if (fp == 1) {
            out[i] = row[0];
            continue;
        }
        for (int v = 0; v * W < nf; v++) {
            const V x = reinterpret_cast<const V*>(row)[v];
            T tmp[W];
            memcpy(tmp, &x, sizeof(V));
#pragma unroll
            for (int c = 0; c < W; c++)
                if (v * W + c < nf) out[(int64_t)(v * W + c) * nt + i] = tmp[c];
        }
    }
}

template <typename T>
void apply_t(MapImpl& M, const T* fields, int nf, T* out, cudaStream_t s) {
    const int64_t ns = M.ns, nt = M.nt;
    constexpr int W = Vec<T>::W;
    int nvec = 1;
    while (nvec * W < nf) nvec <<= 1;   // power-of-two vectors per row
    const int fp = nf == 1 ? 1 : nvec * W;
    DBuf fs(sizeof(T) * fp * std::max<int64_t>(ns, 1), s);
    DBuf stage(sizeof(T) * fp * std::max<int64_t>(nt, 1), s);
    if (ns > 0) {
        PCMS_TRACE("apply_fields_to_sorted", s);
        k_fields_to_sorted<T><<<blocks_for(ns, 256), 256, 0, s>>>(fields, nf, fp, ns,
                                                                  M.src.inv.as<int32_t>(), fs.as<T>());
    }
    if (nt > 0) {
        PCMS_TRACE("apply_spmm", s);
        const int64_t* off = M.offsets.as<int64_t>();
        const int32_t* rc = M.counts.as<int32_t>();
        const int32_t* cols = M.cols.as<int32_t>();
        const T* vals = M.vals.as<T>();
        const int8_t* st = M.status.as<int8_t>();
        DBuf ctr(sizeof(unsigned long long), s);
        unsigned long long* next = ctr.as<unsigned long long>();
        PCMS_CU(cudaMemsetAsync(next, 0, sizeof(unsigned long long), s));
        int nv = fp / W;
        T* fsp = fs.as<T>();
        T* stp = stage.as<T>();
        if (fp == 1) k_spmm_1<T><<<spmm_blocks(k_spmm_1<T>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
        else if constexpr (std::is_same<T, float>::value) {
            if (nv == 1) k_spmm_q<1><<<spmm_blocks(k_spmm_q<1>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
            else if (nv == 2) k_spmm_q<2><<<spmm_blocks(k_spmm_q<2>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
            else if (nv == 4) k_spmm_q<4><<<spmm_blocks(k_spmm_q<4>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
            else fail(PCMS_ERR_INVALID_ARG, "internal: field padding");
        }
        else if (nv == 1) k_spmm_vec<T, 1><<<spmm_blocks(k_spmm_vec<T, 1>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
        else if (nv == 2) k_spmm_vec<T, 2><<<spmm_blocks(k_spmm_vec<T, 2>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
        else if (nv == 4) k_spmm_vec<T, 4><<<spmm_blocks(k_spmm_vec<T, 4>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
        else if (nv == 8) k_spmm_vec<T, 8><<<spmm_blocks(k_spmm_vec<T, 8>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fsp, st, stp, next);
        else {
            fail(PCMS_ERR_INVALID_ARG, "internal: field padding");
        }
        PCMS_LAUNCH_CHECK("k_spmm");
    }
    if (nt > 0) {
        PCMS_TRACE("apply_stage_to_caller", s);
        k_stage_to_caller<T><<<blocks_for(nt, 256), 256, 0, s>>>(stage.as<T>(), fp, nf, nt,
                                                                 M.tgt.inv.as<int32_t>(), out);
    }
    PCMS_LAUNCH_CHECK("apply");
    if (M.qr_n > 0) {
        PCMS_TRACE("apply_qr_rows", s);
        PCMS_CU(qr_apply(M, fields, nf, out, s));
    }
}

// The same three kernels as apply_t, with caller-provided scratch: fs needs ns*fp and stage
// nt*fp elements. Nothing is allocated or traced. Each launch is checked on its own, so an
// error returned here is one of these launches; *where names it. The caller makes sure no
// earlier error is pending on the thread before calling (it would otherwise surface here).
template <typename T>
cudaError_t apply_with_scratch_t(const MapImpl& M, const T* fields, int nf, T* out, T* fs,
                                 T* stage, unsigned long long* next, cudaStream_t s,
                                 const char** where) {
    const int64_t ns = M.ns, nt = M.nt;
    constexpr int W = Vec<T>::W;
    int nvec = 1;
    while (nvec * W < nf) nvec <<= 1;
    const int fp = nf == 1 ? 1 : nvec * W;
    cudaError_t e = cudaSuccess;
    if (ns > 0) {
        k_fields_to_sorted<T><<<blocks_for(ns, 256), 256, 0, s>>>(fields, nf, fp, ns,
                                                                  M.src.inv.as<int32_t>(), fs);
        if ((e = cudaGetLastError()) != cudaSuccess) { *where = "k_fields_to_sorted"; return e; }
    }
    if (nt > 0) {
        const int64_t* off = M.offsets.as<int64_t>();
        const int32_t* rc = M.counts.as<int32_t>();
        const int32_t* cols = M.cols.as<int32_t>();
        const T* vals = M.vals.as<T>();
        const int8_t* st = M.status.as<int8_t>();
        if ((e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), s)) != cudaSuccess) {
            *where = "cudaMemsetAsync (row-chunk counter)";
            return e;
        }
        const int nv = fp / W;
        if (fp == 1) k_spmm_1<T><<<spmm_blocks(k_spmm_1<T>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
        else if constexpr (std::is_same<T, float>::value) {
            if (nv == 1) k_spmm_q<1><<<spmm_blocks(k_spmm_q<1>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
            else if (nv == 2) k_spmm_q<2><<<spmm_blocks(k_spmm_q<2>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
            else k_spmm_q<4><<<spmm_blocks(k_spmm_q<4>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
        }
        else if (nv == 1) k_spmm_vec<T, 1><<<spmm_blocks(k_spmm_vec<T, 1>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
        else if (nv == 2) k_spmm_vec<T, 2><<<spmm_blocks(k_spmm_vec<T, 2>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
        else if (nv == 4) k_spmm_vec<T, 4><<<spmm_blocks(k_spmm_vec<T, 4>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
        else k_spmm_vec<T, 8><<<spmm_blocks(k_spmm_vec<T, 8>, nt), 256, 0, s>>>(nt, off, rc, cols, vals, fs, st, stage, next);
        if ((e = cudaGetLastError()) != cudaSuccess) { *where = "k_spmm"; return e; }
        k_stage_to_caller<T><<<blocks_for(nt, 256), 256, 0, s>>>(stage, fp, nf, nt,
                                                                 M.tgt.inv.as<int32_t>(), out);
        if ((e = cudaGetLastError()) != cudaSuccess) { *where = "k_stage_to_caller"; return e; }
        if ((e = qr_apply(M, fields, nf, out, s)) != cudaSuccess) { *where = "k_qr_apply"; return e; }
    }
    return cudaSuccess;
}

// export: row lengths in caller order, scan, then a warp per row copies (col, val)
__global__ void k_export_len(int64_t nt, const int32_t* __restrict__ inv_t,
                             const int32_t* __restrict__ cnt, int32_t* __restrict__ len) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x)
        len[i] = cnt[inv_t[i]];
}

template <typename T>
__global__ void k_export_rows(int64_t nt, const int32_t* __restrict__ inv_t,
                              const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                              const int32_t* __restrict__ cols,
                              const T* __restrict__ vals, const int32_t* __restrict__ perm_s,
                              const int8_t* __restrict__ st, const int32_t* __restrict__ kx,
                              const int64_t* __restrict__ off_out, int32_t* __restrict__ cols_out,
                              double* __restrict__ vals_out, int8_t* __restrict__ st_out,
                              int32_t* __restrict__ kx_out, int kadd) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nt;
         i += nwarps) {
        const int64_t p = inv_t[i];
        const int64_t a = off[p], b = a + cnt[p], o = off_out[i];
        for (int64_t e = a + lane; e < b; e += 32) {
            cols_out[o + (e - a)] = perm_s[cols[e]];
            if (vals_out) vals_out[o + (e - a)] = (double)vals[e];
        }
        if (lane == 0) {
            if (st_out) st_out[i] = st[p];
            if (kx_out) kx_out[i] = kx[p] + kadd;
        }
    }
}

__global__ void k_export_status(int64_t nt, const int32_t* __restrict__ inv_t,
                                const int8_t* __restrict__ st, const int32_t* __restrict__ kx,
                                int8_t* __restrict__ st_out, int32_t* __restrict__ kx_out,
                                int kadd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = inv_t[i];
        if (st_out) st_out[i] = st[p];
        if (kx_out) kx_out[i] = kx[p] + kadd;
    }
}

}  // namespace

int apply_fp_f32(int nf) {
    int nvec = 1;
    while (nvec * 4 < nf) nvec <<= 1;
    return nf == 1 ? 1 : nvec * 4;
}

void fields_to_sorted_f32(const MapImpl& M, const float* fields, int nf, int fp, float* fs,
                          cudaStream_t s) {
    if (M.ns <= 0) return;
    PCMS_TRACE("apply_fields_to_sorted", s);
    k_fields_to_sorted<float><<<blocks_for(M.ns, 256), 256, 0, s>>>(fields, nf, fp, M.ns,
                                                                    M.src.inv.as<int32_t>(), fs);
    PCMS_LAUNCH_CHECK("fields_to_sorted");
}

void stage_to_caller_f32(const MapImpl& M, const float* stage, int fp, int nf, float* out,
                         cudaStream_t s) {
    if (M.nt <= 0) return;
    PCMS_TRACE("apply_stage_to_caller", s);
    k_stage_to_caller<float><<<blocks_for(M.nt, 256), 256, 0, s>>>(stage, fp, nf, M.nt,
                                                                   M.tgt.inv.as<int32_t>(), out);
    PCMS_LAUNCH_CHECK("stage_to_caller");
}

void mls_apply(MapImpl& M, const void* fields, int nf, void* out, cudaStream_t s) {
    if (M.P.prec == PCMS_MIXED) {
        TuneEntry e;
        if (M.P.dim <= 3 && tune_lookup(M.P.dim, M.P.degree, true, 3, nf, &e) && e.apply_form == 1)
            return mls_apply_tc(M, (const float*)fields, nf, (float*)out, s);
        apply_t<float>(M, (const float*)fields, nf, (float*)out, s);
    } else {
        apply_t<double>(M, (const double*)fields, nf, (double*)out, s);
    }
}

int64_t apply_scratch_bytes(const MapImpl& M, int nf) {
    const int W = M.P.prec == PCMS_MIXED ? 4 : 2;
    const int64_t elem = M.P.prec == PCMS_MIXED ? 4 : 8;
    int nvec = 1;
    while (nvec * W < nf) nvec <<= 1;
    const int64_t fp = nf == 1 ? 1 : nvec * W;
    const int64_t fs = (M.ns * fp * elem + 255) / 256 * 256;   // stage starts 256-aligned
    const int64_t st = (M.nt * fp * elem + 255) / 256 * 256;   // then the row-chunk counter
    return fs + st + 256;
}

cudaError_t mls_apply_with_scratch(const MapImpl& M, const void* fields, int nf, void* out,
                                   void* scratch, cudaStream_t s, const char** where) {
    const int64_t elem = M.P.prec == PCMS_MIXED ? 4 : 8;
    const int W = M.P.prec == PCMS_MIXED ? 4 : 2;
    int nvec = 1;
    while (nvec * W < nf) nvec <<= 1;
    const int64_t fp = nf == 1 ? 1 : nvec * W;
    char* fs = (char*)scratch;
    char* stage = fs + (M.ns * fp * elem + 255) / 256 * 256;
    auto* next = (unsigned long long*)(stage + (M.nt * fp * elem + 255) / 256 * 256);
    if (M.P.prec == PCMS_MIXED)
        return apply_with_scratch_t<float>(M, (const float*)fields, nf, (float*)out, (float*)fs,
                                           (float*)stage, next, s, where);
    return apply_with_scratch_t<double>(M, (const double*)fields, nf, (double*)out,
                                        (double*)fs, (double*)stage, next, s, where);
}

void mls_export(MapImpl& M, int64_t* offsets, int32_t* cols, double* vals, int8_t* status,
                int32_t* kexp, cudaStream_t s) {
    const int64_t nt = M.nt;
    if (offsets == nullptr) {
        if (nt > 0 && (status || kexp))
            k_export_status<<<blocks_for(nt, 256), 256, 0, s>>>(nt, M.tgt.inv.as<int32_t>(),
                                                                M.status.as<int8_t>(),
                                                                M.kexp.as<int32_t>(), status, kexp,
                                                                M.P.kbase);
        PCMS_LAUNCH_CHECK("export");
        return;
    }
    DBuf len(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    if (nt > 0)
        k_export_len<<<blocks_for(nt, 256), 256, 0, s>>>(nt, M.tgt.inv.as<int32_t>(),
                                                         M.counts.as<int32_t>(), len.as<int32_t>());
    exclusive_scan<int64_t>(len.as<int32_t>(), offsets, nt, s);
    if (nt > 0) {
        int blocks = blocks_for(nt * 32, 256, 16);
        if (M.P.prec == PCMS_MIXED)
            k_export_rows<float><<<blocks, 256, 0, s>>>(
                nt, M.tgt.inv.as<int32_t>(), M.offsets.as<int64_t>(), M.counts.as<int32_t>(),
                M.cols.as<int32_t>(), M.vals.as<float>(), M.src.perm.as<int32_t>(), M.status.as<int8_t>(),
                M.kexp.as<int32_t>(), offsets, cols, vals, status, kexp, M.P.kbase);
        else
            k_export_rows<double><<<blocks, 256, 0, s>>>(
                nt, M.tgt.inv.as<int32_t>(), M.offsets.as<int64_t>(), M.counts.as<int32_t>(),
                M.cols.as<int32_t>(), M.vals.as<double>(), M.src.perm.as<int32_t>(), M.status.as<int8_t>(),
                M.kexp.as<int32_t>(), offsets, cols, vals, status, kexp, M.P.kbase);
        qr_export(M, offsets, cols, vals, s);
    }
    PCMS_LAUNCH_CHECK("export");
}

}  // namespace pcms
