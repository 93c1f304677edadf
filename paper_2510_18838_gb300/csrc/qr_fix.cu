// qr_fix.cu -- the Householder-QR pass of the general MLS path (qr.cuh) for targets whose
// FP64 normal equations are too ill-conditioned for the stated accuracy: one-shot transfers
// get those targets' values replaced; cached operators keep an FP64 side table of those
// rows, applied after the sparse product (and used by the export).
#include <algorithm>

#include "qr.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

constexpr int QF_WARPS = 4;

struct QrFixArgs {
    Grid g;
    const int32_t* cell_start;
    const double* sx64;       // [dim][ns] sorted sources
    int64_t ns;
    const int32_t* perm_s;    // sorted source -> caller index
    const double* tx64;       // [dim][nt] sorted targets
    int64_t nt;
    const int32_t* perm_t;    // sorted target -> caller index
    const int32_t* kexp;      // per sorted target: radius doublings
    double radius;
    int weight;
    const int32_t* list;      // sorted targets
    const int32_t* n_list;
    int cap;                  // map mode: side-table entries
    // one-shot: fields [nf][ns] and out [nf][nt] in caller order (float or double)
    const void* fields;
    int nf;
    void* out;
    int8_t* status_caller;    // or null
    // map: status (sorted) and the side table, QR_MAX entries per listed target
    int8_t* status_sorted;
    int32_t* qc;              // sorted source positions
    double* qv;               // operator values
    int32_t* qn;              // entries used (-1: none, the row stays as assembled)
};

template <int DIM, int DEG, typename T, bool MAP>
__global__ void __launch_bounds__(QF_WARPS * 32) k_qr_fix(QrFixArgs A) {
    constexpr int M = mono_count(DIM, DEG);
    __shared__ QrSpace<M> ws[QF_WARPS];
    __shared__ int32_t jl[QF_WARPS][QR_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int n = *A.n_list;
    if (MAP) n = min(n, A.cap);
    for (int e = blockIdx.x * QF_WARPS + w; e < n; e += gridDim.x * QF_WARPS) {
        const int64_t t = A.list[e];
        double tx[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < DIM; d++) tx[d] = A.tx64[d * A.nt + t];
        const int k = A.kexp ? A.kexp[t] : 0;
        const double r = ldexp(A.radius, k);
        const int cnt = qr_collect<DIM>(A.g, A.cell_start, A.sx64, A.ns, tx, r, r * r, A.weight,
                                        jl[w], QR_MAX, lane);
        if (MAP && lane == 0) A.qn[e] = -1;
        if (cnt < M) continue;   // over the cap: the assembled row stands
        double n0, n1;
        const bool ok = qr_row<DIM, DEG>(A.sx64, A.ns, jl[w], cnt, tx, r, A.weight, ws[w], lane, n0, n1);
        const int j0 = lane < cnt ? jl[w][lane] : 0;
        const int j1 = lane + 32 < cnt ? jl[w][lane + 32] : 0;
        if constexpr (MAP) {
            if (!ok) {
                if (lane == 0) A.status_sorted[t] = PCMS_TARGET_ILL_CONDITIONED;
                continue;
            }
            int32_t* qc = A.qc + (int64_t)e * QR_MAX;
            double* qv = A.qv + (int64_t)e * QR_MAX;
            if (lane < cnt) {
                qc[lane] = j0;
                qv[lane] = n0;
            }
            if (lane + 32 < cnt) {
                qc[lane + 32] = j1;
                qv[lane + 32] = n1;
            }
            __syncwarp();
            if (lane == 0) A.qn[e] = cnt;
        } else {
            const int64_t tc = A.perm_t[t];
            const int s0 = lane < cnt ? A.perm_s[j0] : 0;
            const int s1 = lane + 32 < cnt ? A.perm_s[j1] : 0;
            const T* F = (const T*)A.fields;
            T* O = (T*)A.out;
            for (int f = 0; f < A.nf; f++) {
                double v = 0.0;
                if (ok) {
                    if (lane < cnt) v += n0 * (double)F[(int64_t)f * A.ns + s0];
                    if (lane + 32 < cnt) v += n1 * (double)F[(int64_t)f * A.ns + s1];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                } else {
                    v = __longlong_as_double(0x7ff8000000000000LL);
                }
                if (lane == 0) O[(int64_t)f * A.nt + tc] = (T)v;
            }
            if (lane == 0 && A.status_caller)
                A.status_caller[tc] = ok ? PCMS_TARGET_OK : PCMS_TARGET_ILL_CONDITIONED;
        }
        __syncwarp();
    }
}

// out[f][caller t] = sum_i qv[e][i] fields[f][caller source of qc[e][i]], in FP64
template <typename T>
__global__ void __launch_bounds__(QF_WARPS * 32) k_qr_apply(int n, const int32_t* __restrict__ list,
                                                            const int32_t* __restrict__ qc,
                                                            const double* __restrict__ qv,
                                                            const int32_t* __restrict__ qn,
                                                            const int8_t* __restrict__ status,
                                                            const int32_t* __restrict__ perm_s,
                                                            const int32_t* __restrict__ perm_t,
                                                            const T* __restrict__ fields, int nf,
                                                            int64_t ns, T* __restrict__ out,
                                                            int64_t nt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = blockIdx.x * QF_WARPS + w; e < n; e += gridDim.x * QF_WARPS) {
        const int cnt = qn[e];
        const int64_t t = list[e];
        const int64_t tc = perm_t[t];
        if (status[t] != PCMS_TARGET_OK) {   // the QR rank test failed: ill-conditioned
            for (int f = lane; f < nf; f += 32) out[(int64_t)f * nt + tc] = (T)__longlong_as_double(0x7ff8000000000000LL);
            continue;
        }
        if (cnt < 0) continue;
        for (int f = 0; f < nf; f++) {
            double v = 0.0;
            for (int i = lane; i < cnt; i += 32)
                v += qv[(int64_t)e * QR_MAX + i] *
                     (double)fields[(int64_t)f * ns + perm_s[qc[(int64_t)e * QR_MAX + i]]];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) out[(int64_t)f * nt + tc] = (T)v;
        }
    }
}

// export: the listed rows' (col, val) pairs replaced by the side table's (same set of
// sources, any order within a row)
__global__ void k_qr_export(int n, const int32_t* __restrict__ list, const int32_t* __restrict__ qc,
                            const double* __restrict__ qv, const int32_t* __restrict__ qn,
                            const int32_t* __restrict__ perm_s, const int32_t* __restrict__ perm_t,
                            const int64_t* __restrict__ off_out, int32_t* __restrict__ cols_out,
                            double* __restrict__ vals_out) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n; e += nw) {
        const int cnt = qn[e];
        if (cnt < 0) continue;
        const int64_t tc = perm_t[list[e]];
        const int64_t o = off_out[tc];
        if (off_out[tc + 1] - o != cnt) continue;   // not the same row (cannot happen)
        for (int i = lane; i < cnt; i += 32) {
            cols_out[o + i] = perm_s[qc[(int64_t)e * QR_MAX + i]];
            if (vals_out) vals_out[o + i] = qv[(int64_t)e * QR_MAX + i];
        }
    }
}

// enough blocks to fill the GPU (the count may only be known on the device): a warp per
// listed target, as many resident blocks as fit, at most one warp per entry when n is known
template <int DIM, int DEG, typename T, bool MAP>
void launch_fix(const QrFixArgs& a, int64_t n_max, cudaStream_t s) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_fix<DIM, DEG, T, MAP>,
                                                      QF_WARPS * 32, 0) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    const int64_t want = (n_max + QF_WARPS - 1) / QF_WARPS;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
    k_qr_fix<DIM, DEG, T, MAP><<<blocks, QF_WARPS * 32, 0, s>>>(a);
}

template <typename T, bool MAP>
void dispatch_fix(int dim, int deg, const QrFixArgs& a, int64_t n_max, cudaStream_t s) {
    if (dim == 2) {
        if (deg == 1) launch_fix<2, 1, T, MAP>(a, n_max, s);
        else launch_fix<2, 2, T, MAP>(a, n_max, s);
    } else {
        if (deg == 1) launch_fix<3, 1, T, MAP>(a, n_max, s);
        else launch_fix<3, 2, T, MAP>(a, n_max, s);
    }
}

QrFixArgs base_args(const Grid& g, const SortedPoints& S, const SortedPoints& Tp,
                    const int32_t* kexp, double radius, int weight, const int32_t* list,
                    const int32_t* n_list) {
    QrFixArgs a{};
    a.g = g;
    a.cell_start = S.cell_start.as<int32_t>();
    a.sx64 = S.x64.as<double>();
    a.ns = S.n;
    a.perm_s = S.perm.as<int32_t>();
    a.tx64 = Tp.x64.as<double>();
    a.nt = Tp.n;
    a.perm_t = Tp.perm.as<int32_t>();
    a.kexp = kexp;
    a.radius = radius;
    a.weight = weight;
    a.list = list;
    a.n_list = n_list;
    return a;
}

}  // namespace

void qr_fix_transfer(int dim, int deg, bool fp64, const Grid& g, const SortedPoints& S,
                     const SortedPoints& Tp, const int32_t* kexp, double radius, int weight,
                     const int32_t* list, const int32_t* n_list, const void* fields, int nf,
                     void* out, int8_t* status, cudaStream_t s) {
    if (deg < 1 || Tp.n == 0) return;   // degree 0: amp = 1, never listed
    QrFixArgs a = base_args(g, S, Tp, kexp, radius, weight, list, n_list);
    a.fields = fields;
    a.nf = nf;
    a.out = out;
    a.status_caller = status;
    PCMS_TRACE("mls_qr_fix", s);
    if (fp64) dispatch_fix<double, false>(dim, deg, a, Tp.n, s);
    else dispatch_fix<float, false>(dim, deg, a, Tp.n, s);
    PCMS_LAUNCH_CHECK("k_qr_fix");
}

void qr_fix_map(MapImpl& M, const int32_t* list, int n, cudaStream_t s) {
    M.qr_n = 0;
    if (n <= 0 || M.P.degree < 1) return;
    M.qr_list.alloc(sizeof(int32_t) * n, s);
    M.qr_cols.alloc(sizeof(int32_t) * (int64_t)n * QR_MAX, s);
    M.qr_vals.alloc(sizeof(double) * (int64_t)n * QR_MAX, s);
    M.qr_cnt.alloc(sizeof(int32_t) * n, s);
    PCMS_CU(cudaMemcpyAsync(M.qr_list.p, list, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    DBuf cnt(sizeof(int32_t), s);
    PCMS_CU(cudaMemcpyAsync(cnt.p, &n, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    QrFixArgs a = base_args(M.g, M.src, M.tgt, M.kexp.as<int32_t>(), M.P.radius, (int)M.P.weight,
                            M.qr_list.as<int32_t>(), cnt.as<int32_t>());
    a.cap = n;
    a.status_sorted = M.status.as<int8_t>();
    a.qc = M.qr_cols.as<int32_t>();
    a.qv = M.qr_vals.as<double>();
    a.qn = M.qr_cnt.as<int32_t>();
    {
        PCMS_TRACE("mls_qr_rows", s);
        dispatch_fix<float, true>(M.P.dim, M.P.degree, a, n, s);
    }
    PCMS_LAUNCH_CHECK("k_qr_fix (map)");
    PCMS_CU(cudaStreamSynchronize(s));   // the count and the host copy above
    M.qr_n = n;
}

cudaError_t qr_apply(const MapImpl& M, const void* fields, int nf, void* out, cudaStream_t s) {
    if (M.qr_n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((M.qr_n + QF_WARPS - 1) / QF_WARPS, num_sms() * 8);
    if (M.P.prec == PCMS_MIXED)
        k_qr_apply<float><<<blocks, QF_WARPS * 32, 0, s>>>(
            M.qr_n, M.qr_list.as<int32_t>(), M.qr_cols.as<int32_t>(), M.qr_vals.as<double>(),
            M.qr_cnt.as<int32_t>(), M.status.as<int8_t>(), M.src.perm.as<int32_t>(),
            M.tgt.perm.as<int32_t>(), (const float*)fields, nf, M.ns, (float*)out, M.nt);
    else
        k_qr_apply<double><<<blocks, QF_WARPS * 32, 0, s>>>(
            M.qr_n, M.qr_list.as<int32_t>(), M.qr_cols.as<int32_t>(), M.qr_vals.as<double>(),
            M.qr_cnt.as<int32_t>(), M.status.as<int8_t>(), M.src.perm.as<int32_t>(),
            M.tgt.perm.as<int32_t>(), (const double*)fields, nf, M.ns, (double*)out, M.nt);
    return cudaGetLastError();
}

void qr_export(const MapImpl& M, const int64_t* off_out, int32_t* cols_out, double* vals_out,
               cudaStream_t s) {
    if (M.qr_n <= 0) return;
    const int blocks = (int)std::min<int64_t>((M.qr_n * 32 + 255) / 256, num_sms() * 8);
    k_qr_export<<<blocks, 256, 0, s>>>(M.qr_n, M.qr_list.as<int32_t>(), M.qr_cols.as<int32_t>(),
                                       M.qr_vals.as<double>(), M.qr_cnt.as<int32_t>(),
                                       M.src.perm.as<int32_t>(), M.tgt.perm.as<int32_t>(), off_out,
                                       cols_out, vals_out);
    PCMS_LAUNCH_CHECK("k_qr_export");
}

}  // namespace pcms
