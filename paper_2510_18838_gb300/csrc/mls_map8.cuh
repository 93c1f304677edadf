// mls_map8.cuh -- the operator walk of small neighbourhoods (mixed path, FP64 path and the
// mixed path's FP64 tier) with the four 8-lane groups of a warp stepping together (Sec.
// 3.2.1, Eq. 1: the moments of G and the columns of the operator rows).
//
// k_assemble with G = 8 lets each group run its own walk: a group pops its compaction ring
// (and runs the moment update, the costly part of a selected pair) as soon as it holds 8
// pairs, so the warp executes the update whenever any of its four groups pops, mostly with
// one or two groups active. Here the warp's control flow is uniform: the four targets of a
// warp are set up together, their candidate streams are stepped in lockstep up to the
// longest, and the rings (32 entries per group) are popped together, when every group holds
// 8 pairs or has ended its stream, or when one ring could overflow on the next step. The
// moment update then runs with all 32 lanes busy in most pops.
//
// Pairs reach the lanes exactly as in k_assemble (ring entry i of a target to lane i mod 8,
// in stream order), so the per-lane sums, the moments and the columns are the same bit for
// bit; only the schedule of the pops differs. Plain sums (FP32 on the mixed path, FP64
// otherwise, where a warp's FP64 instructions take the narrow FP64 pipe whatever their
// active lanes, so the divergent pops cost even more), MODE_MAP, one pass or a given row (the
// second walk of rows that did not fit the stage), optional target list and, for the FP64
// form, the list's re-centred bases. Measured on 1M -> 1M operators, FP64: 3D quadratic
// 22.5 -> 16.4 ms, 3D linear 9.1 -> 7.2 ms.
#pragma once

#include "mls_kernels.cuh"

namespace pcms {

// Sizes of the walk: 8 lanes per target, 4 targets per warp, 8 warps per block.
struct Map8 {
    static constexpr int G = 8, GPW = 4;
    static constexpr int QCAP = 4 * G;   // ring entries per group (a power of two)
    static constexpr int STG = 384;      // staged columns per group (one-pass rows)
    template <int DIM>
    static constexpr int RPL = DIM == 3 ? 4 : 1;   // rows set up per lane and batch
};

// Shared memory of one block (one copy for both weight instantiations of the body). Ring
// entries are (offsets, payload) as float4 (mixed) or double4 (FP64).
template <int DIM, bool MIXED>
struct Map8Smem {
    using QE = typename QEntry<typename std::conditional<MIXED, float, double>::type>::type;
    QE q[8][Map8::GPW * Map8::QCAP];
    int rowa[8][Map8::GPW * Map8::G * Map8::RPL<DIM>];
    int rowe[8][Map8::GPW * Map8::G * Map8::RPL<DIM>];
    int32_t stg[8 * Map8::GPW * Map8::STG];
};

template <int DIM, int DEG, bool MIXED, int WK>
__device__ __forceinline__ void map8_body(const AsmArgs& A, Map8Smem<DIM, MIXED>& S) {
    using T = typename std::conditional<MIXED, float, double>::type;
    using QE = typename Map8Smem<DIM, MIXED>::QE;
    constexpr int G = Map8::G, GPW = Map8::GPW, QCAP = Map8::QCAP, STG = Map8::STG;
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int NACCP = round_up4(NM);
    constexpr int RPL = Map8::RPL<DIM>;
    constexpr int RB = G * RPL;
    constexpr unsigned FULL = 0xffffffffu;

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gi = lane >> 3, gl = lane & 7;
    const unsigned gmask = 0xffu << (gi * G);
    const unsigned lt = (1u << lane) - 1u;
    QE* q = &S.q[wib][gi * QCAP];
    int* rA = &S.rowa[wib][gi * RB];
    int* rE = &S.rowe[wib][gi * RB];
    int32_t* stg = &S.stg[(wib * GPW + gi) * STG];
    const Grid& g = A.g;
    const bool one_pass = A.one_pass != 0;
    const int64_t nwork = A.list ? (int64_t)(*A.n_list) : A.nt;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5) * GPW;

    for (int64_t wb = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GPW; wb < nwork;
         wb += wstride) {   // uniform over the warp
        const int64_t wk = wb + gi;
        const bool act = wk < nwork;
        const int64_t t = act ? (A.list ? (int64_t)A.list[wk] : wk) : 0;
        long long ct[3] = {0, 0, 0};
        float fr[3] = {0.f, 0.f, 0.f};
        float thi[3] = {0.f, 0.f, 0.f}, tlo[3] = {0.f, 0.f, 0.f};
        double tx[3] = {0.0, 0.0, 0.0};   // FP64 walk: the target's coordinates
        T bcv[4] = {T(0), T(0), T(0), T(1)};
        bool recentred = false;           // FP64 list mode: a re-centred basis per entry
        int k = 0;
        int64_t row_off = 0, row_len = 0;
        if (act) {
            if constexpr (!MIXED) {
#pragma unroll
                for (int d = 0; d < DIM; d++) tx[d] = A.tx64[d * A.nt + t];
                if (A.basis) {
                    const float4 bb = A.basis[wk];
                    bcv[0] = bb.x;
                    bcv[1] = bb.y;
                    bcv[2] = bb.z;
                    bcv[3] = bb.w;
                    recentred = true;
                }
            }
            const int4 c4 = A.tcell[t];
            const float4 f4 = A.tfrac[t];
            ct[0] = c4.x;
            ct[1] = c4.y;
            ct[2] = c4.z;
            fr[0] = f4.x;
            fr[1] = f4.y;
            fr[2] = f4.z;
            if constexpr (MIXED) load_hilo<DIM>(A.thl0, A.thl1, t, thi, tlo);
            k = A.kexp_in ? A.kexp_in[t] : 0;
            if (!one_pass && A.cols) {   // the first walk fixed the row
                row_off = A.offsets[t];
                row_len = A.counts[t];
            }
        }
        const double r = A.lv.r[k];
        const double r2 = A.lv.r2[k];
        const double r2_in = r2 * (1.0 - 9.094947017729282e-13);
        const float r2f = A.lv.r2f[k];
        const T inv_r = MIXED ? (T)A.lv.inv_rf[k] : (T)A.lv.inv_r[k];
        const float R0 = A.lv.rcell[k];
        const float mg = 1e-3f + R0 * 1e-6f;
        const float RR = R0 + mg;
        long long z0 = 0, z1 = 0;
        if (DIM == 3) {
            z0 = max((long long)__float2int_rd(fr[2] - RR), -ct[2]);
            z1 = min((long long)__float2int_rd(fr[2] + RR), (long long)g.n[2] - 1 - ct[2]);
        }
        const long long y0 = max((long long)__float2int_rd(fr[1] - RR), -ct[1]);
        const long long y1 =
            min((long long)__float2int_rd(fr[1] + RR), (long long)g.n[1] - 1 - ct[1]);
        const long long ny = y1 >= y0 ? y1 - y0 + 1 : 0;
        long long nrows = ny * (DIM == 3 ? (z1 >= z0 ? z1 - z0 + 1 : 0) : 1);
        if (!act) nrows = 0;

        T acc[NM];
#pragma unroll
        for (int i = 0; i < NM; i++) acc[i] = T(0);
        int qn = 0, head = 0, cnt = 0;
        int64_t written = 0;

        // pops G ring entries into the lanes' sums and the row's columns
        auto pop = [&](int n) {
            if (gl < n) {
                const QE e = q[(head + gl) & (QCAP - 1)];
                const T edx[3] = {e.x, e.y, e.z};
                accumulate<DIM, DEG, MODE_MAP, T, NM, WK>(acc, edx, e.w, A.weight, inv_r,
                                                          recentred ? bcv : nullptr);
                const int32_t j = unpack_index(e.w);
                if (one_pass) {
                    if (written + gl < STG) stg[written + gl] = j;
                } else if (A.cols && written + gl < row_len) {
                    A.cols[row_off + written + gl] = j;
                }
            }
            written += n;
            head = (head + n) & (QCAP - 1);
            qn -= n;
        };

        const int nb = __reduce_max_sync(FULL, (int)((nrows + RB - 1) / RB));
        for (int bi = 0; bi < nb; bi++) {
            const long long row0 = (long long)bi * RB;
            int64_t cs0[RPL], cs1[RPL];
            bool live[RPL];
#pragma unroll
            for (int i = 0; i < RPL; i++) {
                const long long rho = row0 + gl * RPL + i;
                int64_t rowbase = 0;
                long long x0 = 0, x1 = 0;
                live[i] = rho < nrows &&
                          row_chord<DIM>(g, ct, fr, RR, mg, y0, z0, ny, rho, rowbase, x0, x1);
                cs0[i] = rowbase + x0;
                cs1[i] = rowbase + x1 + 1;
            }
            int ra[RPL], rl[RPL], lsum = 0;
#pragma unroll
            for (int i = 0; i < RPL; i++) {
                ra[i] = live[i] ? A.cell_start[cs0[i]] : 0;
                rl[i] = live[i] ? A.cell_start[cs1[i]] - ra[i] : 0;
                lsum += rl[i];
            }
            int incl = lsum;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o, G);
                if (gl >= o) incl += v;
            }
            const int total = __shfl_sync(FULL, incl, G - 1, G);
            int e = incl - lsum;
#pragma unroll
            for (int i = 0; i < RPL; i++) {
                e += rl[i];
                rA[gl * RPL + i] = ra[i];
                rE[gl * RPL + i] = e;
            }
            __syncwarp();
            const int tmax = __reduce_max_sync(FULL, total);

            int rcur = 0, pos = gl, pend = 0, jn = 0;
            Cand<MIXED, DIM, float, false> cn{};
            bool vn = pos < total;
            if (vn) {
                while (rE[rcur] <= pos) ++rcur;
                pend = rE[rcur];
                jn = rA[rcur] + pos - (rcur ? rE[rcur - 1] : 0);
                cn.load(A, jn);
            }
            for (int p0 = 0; p0 < tmax; p0 += G) {
                const bool v = vn;
                const int j = jn;
                const Cand<MIXED, DIM, float, false> c = cn;
                pos += G;
                vn = pos < total;
                if (vn) {
                    if (pos < pend) {
                        jn += G;
                    } else {   // pos >= rE[rcur]: the loop moves rcur at least once
                        while (rE[rcur] <= pos) ++rcur;
                        pend = rE[rcur];
                        jn = rA[rcur] + pos - rE[rcur - 1];
                    }
                    cn.load(A, jn);
                }
                bool in = false;
                T ddx = T(0), ddy = T(0), ddz = T(0);
                if (!MIXED && v) {   // FP64 walk: the definition's squared distance
                    const double e0 = __dsub_rn(c.x[0], tx[0]);
                    const double e1 = __dsub_rn(c.x[1], tx[1]);
                    double d2 = __dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1));
                    double e2 = 0.0;
                    if (DIM == 3) {
                        e2 = __dsub_rn(c.x[2], tx[2]);
                        d2 = __dadd_rn(d2, __dmul_rn(e2, e2));
                    }
                    in = select64(A.weight, d2, r, r2, r2_in);
                    ddx = (T)e0;
                    ddy = (T)e1;
                    ddz = (T)e2;
                }
                if (MIXED && v) {
                    const float4 h0 = c.h0;
                    const float2 h1 = c.h1;
                    if (DIM == 2) {
                        ddx = (h0.x - thi[0]) + (h0.z - tlo[0]);
                        ddy = (h0.y - thi[1]) + (h0.w - tlo[1]);
                    } else {
                        ddx = (h0.x - thi[0]) + (h0.w - tlo[0]);
                        ddy = (h0.y - thi[1]) + (h1.x - tlo[1]);
                        ddz = (h0.z - thi[2]) + (h1.y - tlo[2]);
                    }
                    float d2f = ddx * ddx + ddy * ddy;
                    if (DIM == 3) d2f += ddz * ddz;
                    int cl;
                    if constexpr (WK == PCMS_WENDLAND_C2)
                        cl = d2f > r2f * (1.0f + MIX_BAND)
                                 ? 0
                                 : (d2f < r2f * (1.0f - MIX_BAND) ? 1 : -1);
                    else
                        cl = classify32(A.weight, d2f, r2f);
                    if (cl < 0) {   // within 2^-16 of the radius: the exact FP64 decision
                        double te[3] = {0.0, 0.0, 0.0};
#pragma unroll
                        for (int d = 0; d < DIM; d++) te[d] = A.tx64[d * A.nt + t];
                        cl = select_exact(A.weight, dist2_exact<DIM>(A.sx64, A.ns, j, te), r, r2);
                    }
                    in = cl != 0;
                }
                const unsigned gb = __ballot_sync(FULL, in) & gmask;
                const int nin = __popc(gb);
                if (in) {
                    const int qp = (head + qn + __popc(gb & lt)) & (QCAP - 1);
                    q[qp] = make_entry<T>(ddx, ddy, ddz, pack_index(j, T(0)));
                }
                qn += nin;
                cnt += nin;
                __syncwarp();
                // Pop together: when every group holds G pairs or has ended this stream, or
                // when a ring could not take another step's G entries.
                const bool ready = qn >= G;
                const bool ended = p0 + G >= total;
                if (__any_sync(FULL, qn > QCAP - G) || __all_sync(FULL, ready || ended)) {
                    if (ready) pop(G);
                    __syncwarp();   // the popped entries are read before they are rewritten
                }
            }
            __syncwarp();   // the row table is rewritten by the next batch
        }
        while (__any_sync(FULL, qn >= G)) {
            if (qn >= G) pop(G);
            __syncwarp();
        }
        if (qn > 0) pop(qn);
        __syncwarp();

#pragma unroll
        for (int i = 0; i < NM; i++) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(FULL, acc[i], o);
        }
        if (act && gl == 0) {
            T* dst = (T*)A.mom + (A.list ? wk : t) * NACCP;
#pragma unroll
            for (int i = 0; i < NACCP; i++) dst[i] = i < NM ? acc[i < NM ? i : 0] : T(0);
            A.counts[t] = cnt;
            if (A.kexp_out) A.kexp_out[t] = k;
            if (!one_pass && A.cols && cnt != row_len) atomicOr(A.err, 1u);
        }
        if (one_pass) {
            // reserve the row, then copy the staged columns (or leave the row to the second walk)
            unsigned long long base = 0;
            if (act && gl == 0) base = atomicAdd(A.nnz_ctr, (unsigned long long)cnt);
            base = __shfl_sync(FULL, base, 0, G);
            const bool fits = cnt <= STG && (int64_t)(base + cnt) <= A.cols_cap;
            if (act && fits)
                for (int i = gl; i < cnt; i += G) A.cols[base + i] = stg[i];
            if (act && gl == 0) {
                A.offsets[t] = (int64_t)base;
                if (!fits) A.redo[atomicAdd(A.n_redo, 1)] = (int32_t)t;
            }
        }
        __syncwarp();   // the ring, row table and stage are reused by the next targets
    }
}

// The block's Map8Smem is dynamic shared memory (the FP64 form's 32-byte ring entries take it
// past the 48 KB of static shared memory).
template <int DIM, int DEG, bool MIXED>
__global__ void __launch_bounds__(256, asm_min_blocks<DIM, DEG, ACC_PLAIN, MIXED, MODE_MAP, 8>())
    k_assemble_map8(AsmArgs A) {
    extern __shared__ __align__(32) unsigned char map8_smem[];
    Map8Smem<DIM, MIXED>& S = *reinterpret_cast<Map8Smem<DIM, MIXED>*>(map8_smem);
    if (A.weight == PCMS_WENDLAND_C2) map8_body<DIM, DEG, MIXED, PCMS_WENDLAND_C2>(A, S);
    else map8_body<DIM, DEG, MIXED, -1>(A, S);
}

template <int DIM, int DEG, bool MIXED>
void launch_map8(const AsmArgs& a, int blocks, cudaStream_t s) {
    constexpr size_t smem = sizeof(Map8Smem<DIM, MIXED>);
    if (smem > 48 * 1024)
        PCMS_CU(cudaFuncSetAttribute(k_assemble_map8<DIM, DEG, MIXED>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_assemble_map8<DIM, DEG, MIXED><<<blocks, 256, smem, s>>>(a);
}

}  // namespace pcms
