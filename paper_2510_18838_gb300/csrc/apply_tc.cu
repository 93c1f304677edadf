// apply_tc.cu -- the multi-field apply of a mixed (FP32) operator on the tensor cores:
// out[t][f] = sum_j N_tj F_jf (Sec. 3.2.1, Eq. 1, applied to up to 16 fields) as BF16 x BF16
// products accumulated in FP32, with a compensated three-term split of both operands.
//
// Each FP32 value x is split into three BF16 terms, x = x_h + x_m + x_l + d with
// x_h = bf16(x), x_m = bf16(x - x_h), x_l = bf16(x - x_h - x_m), |d| <= 2^-24 |x| (24 of the
// 24 significand bits). The product N F is the sum of the six term products of order <= 2,
//   N_h F_h + (N_h F_m + N_m F_h) + (N_h F_l + N_m F_m + N_l F_h),
// the first being the plain BF16 product and the rest its residual correction; the omitted
// terms are below 3 2^-24 |N F|, so the result has the accuracy of an FP32 apply. The three
// orders go to separate FP32 accumulators, added at the end (the tensor cores' accumulation
// aligns each group of products to the running sum, which would cut the small correction
// terms if they were added into it).
//
// Mapping onto mma.sync.m16n8k16 (BF16 inputs, FP32 accumulators): a warp takes 16
// consecutive targets (cell-sorted, so their sources overlap in L1/L2) and walks the
// concatenation of their nonzeros 16 at a time ("slots"). A = the 16 x 16 block of operator
// values, A[g][k] = N of slot k if slot k belongs to target g, else 0 (built in registers);
// B = the 16 slots' field rows (16 fields), gathered from the pre-split BF16 field planes
// into shared memory by cp.async, double buffered, and read with ldmatrix.trans. Two MMAs
// (fields 0-7, 8-15) per term product, twelve per 16 slots. The block-diagonal A makes 15 of
// every 16 multiply-adds zero: the apply is a sparse contraction, and the tensor cores only
// replace the CUDA-core multiply-adds, not the gathers.
#include <cuda_bf16.h>

#include <algorithm>

#include "pcms_internal.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

constexpr int TC_WARPS = 4;
constexpr int TC_FIELDS = 16;

__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m,
                                       __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// caller-order fields [nf][ns] -> three BF16 planes [3][ns][16] in sorted source order
__global__ void k_fields_bf16x3(const float* __restrict__ f, int nf, int64_t ns,
                                const int32_t* __restrict__ inv, __nv_bfloat16* __restrict__ fs3) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = inv[i];
        uint32_t w[3][8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(2 * q < nf ? f[(int64_t)(2 * q) * ns + i] : 0.f, h0, m0, l0);
            split3(2 * q + 1 < nf ? f[(int64_t)(2 * q + 1) * ns + i] : 0.f, h1, m1, l1);
            w[0][q] = pack2(h0, h1);
            w[1][q] = pack2(m0, m1);
            w[2][q] = pack2(l0, l1);
        }
#pragma unroll
        for (int sp = 0; sp < 3; sp++) {
            uint4* dst = reinterpret_cast<uint4*>(fs3 + ((int64_t)sp * ns + row) * TC_FIELDS);
            dst[0] = make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
            dst[1] = make_uint4(w[sp][4], w[sp][5], w[sp][6], w[sp][7]);
        }
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;   // 0: the 16 bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* smem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(sa));
}

struct TcWarpSmem {
    __nv_bfloat16 pan[2][3][16][TC_FIELDS];   // double-buffered B panels, [split][slot][field]
    int32_t end[16];                          // the tile's rows: slot end (exclusive)
    int64_t off[16];                          // and row start minus its first slot
    int32_t own[2][16];                       // per buffered slot: owning row (-1: none)
    float val[2][16];                         // and operator value
};

// One warp per tile of 16 targets, tiles taken from a counter.
__global__ void __launch_bounds__(TC_WARPS * 32) k_spmm_tc(
    int64_t nt, const int64_t* __restrict__ offs, const int32_t* __restrict__ cnt,
    const int32_t* __restrict__ cols, const float* __restrict__ vals,
    const __nv_bfloat16* __restrict__ fs3, int64_t ns, const int8_t* __restrict__ status,
    float* __restrict__ stage, unsigned long long* next) {
    __shared__ __align__(128) TcWarpSmem sm_all[TC_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TcWarpSmem& S = sm_all[w];
    const unsigned full = 0xffffffffu;
    const int g = lane >> 2, c = lane & 3;
    const int64_t ntiles = (nt + 15) / 16;
    for (;;) {
        long long tile = 0;
        if (lane == 0) tile = (long long)atomicAdd(next, 1ull);
        tile = __shfl_sync(full, tile, 0);
        if (tile >= ntiles) break;
        const int64_t t0 = tile * 16;
        // the tile's rows: slot ranges by a prefix sum over the 16 row lengths
        int len = 0;
        int64_t o = 0;
        if (lane < 16 && t0 + lane < nt) {
            len = cnt[t0 + lane];
            o = offs[t0 + lane];
        }
        int incl = len;
#pragma unroll
        for (int d = 1; d < 16; d <<= 1) {
            const int v = __shfl_up_sync(full, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(full, incl, 15);
        if (lane < 16) {
            S.end[lane] = incl;
            S.off[lane] = o - (incl - len);   // row start minus its first slot
        }
        __syncwarp();
        // stage slots [k0, k0 + 16) into buffer b: lanes 0-15 find their slot's row, value and
        // column; then 96 cp.async of 16 bytes (3 splits x 16 slots x 2 halves), 3 per lane
        auto stage_slots = [&](int k0, int b) {
            int col = 0;
            if (lane < 16) {
                const int k = k0 + lane;
                int r = -1;
                float v = 0.f;
                if (k < total) {
                    int a = 0, e = 15;   // the first row whose end is above k
                    while (a < e) {
                        const int mid = (a + e) >> 1;
                        if (S.end[mid] > k) e = mid;
                        else a = mid + 1;
                    }
                    r = a;
                    const int64_t idx = (int64_t)S.off[r] + k;
                    col = cols[idx];
                    v = vals[idx];
                }
                S.own[b][lane] = r;
                S.val[b][lane] = v;
            }
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const int id = lane + 32 * q;   // 0..95
                const int sp = id >> 5, slot = (id & 31) >> 1, half = id & 1;
                const int cs = __shfl_sync(full, col, slot);
                const bool valid = k0 + slot < total;
                const __nv_bfloat16* src = fs3 + ((int64_t)sp * ns + (valid ? cs : 0)) * TC_FIELDS + half * 8;
                cp_async16(&S.pan[b][sp][slot][half * 8], src, valid);
            }
            asm volatile("cp.async.commit_group;\n" ::);
        };
        // three accumulators per field half: the BF16 product (order 0) and the corrections
        // of order 1 and 2, summed at the end, so that the tensor cores' accumulation never
        // adds the small correction terms into the large running sum
        float acc[3][2][4];
#pragma unroll
        for (int o = 0; o < 3; o++)
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[o][h][i] = 0.f;
        if (total > 0) stage_slots(0, 0);
        for (int k0 = 0, b = 0; k0 < total; k0 += 16, b ^= 1) {
            if (k0 + 16 < total) {
                stage_slots(k0 + 16, b ^ 1);
                asm volatile("cp.async.wait_group 1;\n" ::);
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::);
            }
            __syncwarp();
            // A: the block-diagonal operator values of these slots, three BF16 terms
            uint32_t A[3][4];
            {
                const int ks[4] = {2 * c, 2 * c + 1, 2 * c + 8, 2 * c + 9};
                __nv_bfloat16 hv[2][4], mv[2][4], lv[2][4];   // [row g / g+8][slot]
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int r = S.own[b][ks[q]];
                    const float v = S.val[b][ks[q]];
                    split3(r == g ? v : 0.f, hv[0][q], mv[0][q], lv[0][q]);
                    split3(r == g + 8 ? v : 0.f, hv[1][q], mv[1][q], lv[1][q]);
                }
                A[0][0] = pack2(hv[0][0], hv[0][1]);
                A[0][1] = pack2(hv[1][0], hv[1][1]);
                A[0][2] = pack2(hv[0][2], hv[0][3]);
                A[0][3] = pack2(hv[1][2], hv[1][3]);
                A[1][0] = pack2(mv[0][0], mv[0][1]);
                A[1][1] = pack2(mv[1][0], mv[1][1]);
                A[1][2] = pack2(mv[0][2], mv[0][3]);
                A[1][3] = pack2(mv[1][2], mv[1][3]);
                A[2][0] = pack2(lv[0][0], lv[0][1]);
                A[2][1] = pack2(lv[1][0], lv[1][1]);
                A[2][2] = pack2(lv[0][2], lv[0][3]);
                A[2][3] = pack2(lv[1][2], lv[1][3]);
            }
            // B: matrix m of ldmatrix = slots (m & 1) * 8 .. + 7, fields (m >> 1) * 8 .. + 7
            uint32_t B[3][4];
            {
                const int m = lane >> 3;
                const int slot = (m & 1) * 8 + (lane & 7);
#pragma unroll
                for (int sp = 0; sp < 3; sp++) ldsm_x4_trans(B[sp], &S.pan[b][sp][slot][(m >> 1) * 8]);
            }
            // the six term products of order <= 2, fields 0-7 (B regs 0, 1) and 8-15 (2, 3)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                mma_bf16(acc[0][h], A[0], B[0][2 * h], B[0][2 * h + 1]);
                mma_bf16(acc[1][h], A[0], B[1][2 * h], B[1][2 * h + 1]);
                mma_bf16(acc[1][h], A[1], B[0][2 * h], B[0][2 * h + 1]);
                mma_bf16(acc[2][h], A[0], B[2][2 * h], B[2][2 * h + 1]);
                mma_bf16(acc[2][h], A[1], B[1][2 * h], B[1][2 * h + 1]);
                mma_bf16(acc[2][h], A[2], B[0][2 * h], B[0][2 * h + 1]);
            }
            __syncwarp();   // buffer b is restaged two steps on
        }
        // D[g][2c..2c+1] and D[g + 8][...] for fields h * 8 + 2c, + 1
        const float nan = __int_as_float(0x7fc00000);
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
            const int64_t t = t0 + g + 8 * rr;
            if (t < nt) {
                const bool ok = status[t] == PCMS_TARGET_OK;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    float2 v = make_float2(acc[0][h][2 * rr] + (acc[1][h][2 * rr] + acc[2][h][2 * rr]),
                                           acc[0][h][2 * rr + 1] + (acc[1][h][2 * rr + 1] + acc[2][h][2 * rr + 1]));
                    if (!ok) v = make_float2(nan, nan);
                    *reinterpret_cast<float2*>(stage + t * TC_FIELDS + h * 8 + 2 * c) = v;
                }
            }
        }
        __syncwarp();
    }
}

__global__ void k_stage16_to_caller(const float* __restrict__ stage, int nf, int64_t nt,
                                    const int32_t* __restrict__ inv_t, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float* row = stage + (int64_t)inv_t[i] * TC_FIELDS;
        for (int f = 0; f < nf; f++) out[(int64_t)f * nt + i] = row[f];
    }
}

int grid_for(int64_t n, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)num_sms() * 32));
}

}  // namespace

void mls_apply_tc(MapImpl& M, const float* fields, int nf, float* out, cudaStream_t s) {
    if (M.P.prec != PCMS_MIXED) fail(PCMS_ERR_INVALID_ARG, "the tensor-core apply needs a mixed map");
    const int64_t ns = M.ns, nt = M.nt;
    DBuf fs3(sizeof(__nv_bfloat16) * 3 * TC_FIELDS * std::max<int64_t>(ns, 1), s);
    DBuf stage(sizeof(float) * TC_FIELDS * std::max<int64_t>(nt, 1), s);
    if (ns > 0) {
        PCMS_TRACE("apply_fields_bf16x3", s);
        k_fields_bf16x3<<<grid_for(ns, 256), 256, 0, s>>>(fields, nf, ns, M.src.inv.as<int32_t>(),
                                                          fs3.as<__nv_bfloat16>());
    }
    PCMS_LAUNCH_CHECK("k_fields_bf16x3");
    if (nt > 0) {
        DBuf ctr(sizeof(unsigned long long), s);
        PCMS_CU(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long), s));
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_tc, TC_WARPS * 32, 0) !=
                cudaSuccess || per_sm < 1) {
            (void)cudaGetLastError();
            per_sm = 1;
        }
        const int64_t tiles = (nt + 15) / 16;
        const int blocks = (int)std::max<int64_t>(
            1, std::min<int64_t>((tiles + TC_WARPS - 1) / TC_WARPS, (int64_t)num_sms() * per_sm));
        {
            PCMS_TRACE("apply_spmm_tc", s);
            k_spmm_tc<<<blocks, TC_WARPS * 32, 0, s>>>(
                nt, M.offsets.as<int64_t>(), M.counts.as<int32_t>(), M.cols.as<int32_t>(),
                M.vals.as<float>(), fs3.as<__nv_bfloat16>(), ns, M.status.as<int8_t>(),
                stage.as<float>(), ctr.as<unsigned long long>());
        }
        PCMS_LAUNCH_CHECK("k_spmm_tc");
        {
            PCMS_TRACE("apply_stage_to_caller", s);
            k_stage16_to_caller<<<grid_for(nt, 256), 256, 0, s>>>(stage.as<float>(), nf, nt,
                                                                   M.tgt.inv.as<int32_t>(), out);
        }
        PCMS_LAUNCH_CHECK("k_stage16_to_caller");
    }
    if (M.qr_n > 0) {
        PCMS_TRACE("apply_qr_rows", s);
        PCMS_CU(qr_apply(M, fields, nf, out, s));
    }
}

}  // namespace pcms
