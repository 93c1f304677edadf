// qr.cuh -- the Householder-QR solve of one target's weighted least-squares fit (Sec. 3.2.1,
// Eq. 1), by one warp, for the targets whose normal equations are too ill-conditioned for
// the stated accuracy.
//
// The assembly kernels solve the normal equations G y = a_t (G = A^T W A), which square the
// condition number of the weighted Vandermonde matrix B = diag(sqrt(w)) A: a fit through
// about m nearly degenerate points (an extrapolating target, a corner of the domain, a
// neighbourhood that is almost a plane for a quadratic basis) loses digits that no precision
// tier of the normal equations recovers. For such targets (those whose conditioning estimate
// amp is still large in FP64) the kernels list the target, and a warp computes, in FP64:
//   B = diag(sqrt(w)) A, rows = the selected sources, columns = the target-centred,
//       radius-scaled graded-lex monomials;
//   B = Q R by Householder reflections, with the rank test of the definition: column k is
//       dependent when |R_kk| <= 1e-7 ||column k of B|| (ill-conditioned: NaN);
//   N = diag(sqrt(w)) Q R^-T e_1, the operator row, so that f(t) = sum_j N_j f_j.
// The error of N then grows with cond(B), not cond(B)^2.
#pragma once

#include "mls_kernels.cuh"

namespace pcms {

constexpr int QR_MAX = 64;   // at most this many neighbours (such fits are small)

// The selected sources of target tx at radius r (sorted positions, any order), collected by
// one warp from the cells within r: every candidate is decided exactly in FP64 (the
// definition's predicate, as every assembly decides it). Returns the count, or -1 if it
// exceeds cap (jl then holds an incomplete list).
template <int DIM>
__device__ __forceinline__ int qr_collect(const Grid& g, const int32_t* __restrict__ cell_start,
                                          const double* __restrict__ sx64, int64_t ns,
                                          const double* tx, double r, double r2, int weight,
                                          int32_t* jl, int cap, int lane) {
    const unsigned full = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    long long c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
    const double R = r * g.inv_h;
    // a ball that spans too many cells (a radius grown many times) is left to the normal
    // equations: its count is far above cap anyway
    if (!(R < 12.0)) return -1;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        const double u = (tx[d] - g.lo[d]) * g.inv_hd(d);
        const double Rd = r * g.inv_hd(d);
        // one cell of margin each side covers the rounding of u and of the cells' keys
        const double a = fmax(floor(u - Rd) - 1.0, 0.0);
        const double b = fmin(floor(u + Rd) + 1.0, (double)(g.n[d] - 1));
        c0[d] = (long long)a;
        c1[d] = (long long)b;
        if (b < a) return 0;
    }
    int cnt = 0;
    for (long long z = c0[2]; z <= c1[2]; z++) {
        for (long long y = c0[1]; y <= c1[1]; y++) {
            const int64_t rowbase = (z * g.n[1] + y) * (int64_t)g.n[0];
            const int a = cell_start[rowbase + c0[0]];
            const int e = cell_start[rowbase + c1[0] + 1];
            for (int p0 = a; p0 < e; p0 += 32) {
                const int j = p0 + lane;
                bool in = false;
                if (j < e) in = select_exact(weight, dist2_exact<DIM>(sx64, ns, j, tx), r, r2);
                const unsigned bal = __ballot_sync(full, in);
                if (in && cnt + __popc(bal & lt) < cap) jl[cnt + __popc(bal & lt)] = j;
                cnt += __popc(bal);
            }
        }
    }
    __syncwarp();
    return cnt > cap ? -1 : cnt;
}

// Per-warp work space of qr_row (shared memory).
template <int M>
struct QrSpace {
    double B[M][QR_MAX];   // column k, row i; rows >= k of column k become v_k
    double sw[QR_MAX];
    double beta[M], rkk[M];
};

// The operator row of a target with the cnt (<= QR_MAX) selected sources jl: on return each
// lane holds N for rows lane and lane + 32 (0 beyond cnt). Returns false when the rank test
// fails (ill-conditioned).
template <int DIM, int DEG>
__device__ __forceinline__ bool qr_row(const double* __restrict__ sx64, int64_t ns, const int32_t* jl,
                                       int cnt, const double* tx, double r, int weight,
                                       QrSpace<mono_count(DIM, DEG)>& W, int lane, double& n0,
                                       double& n1) {
    constexpr int M = mono_count(DIM, DEG);
    const unsigned full = 0xffffffffu;
    auto wsum = [&](double v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
        return v;
    };
    const double inv_r = 1.0 / r;
    for (int i = lane; i < QR_MAX; i += 32) {
        double swi = 0.0;
        double a[M];
#pragma unroll
        for (int k = 0; k < M; k++) a[k] = 0.0;
        if (i < cnt) {
            const int j = jl[i];
            double dx[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int d = 0; d < DIM; d++) dx[d] = __dsub_rn(sx64[d * ns + j], tx[d]);
            double d2 = __dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1]));
            if (DIM == 3) d2 = __dadd_rn(d2, __dmul_rn(dx[2], dx[2]));
            swi = sqrt(weight_value<double>(weight, sqrt(d2) / r));
            const double u[3] = {dx[0] * inv_r, dx[1] * inv_r, dx[2] * inv_r};
            a[0] = 1.0;
            sfor<M - 1>([&](auto I) {
                constexpr int p = decltype(I)::value + 1;
                a[p] = a[mono_parent(DIM, p)] * u[mono_var(DIM, p)];
            });
        }
        W.sw[i] = swi;
#pragma unroll
        for (int k = 0; k < M; k++) W.B[k][i] = swi * a[k];
    }
    __syncwarp();
    double cn[M];
#pragma unroll
    for (int k = 0; k < M; k++)
        cn[k] = sqrt(wsum(W.B[k][lane] * W.B[k][lane] + W.B[k][lane + 32] * W.B[k][lane + 32]));
#pragma unroll
    for (int k = 0; k < M; k++) {
        const double x0 = lane >= k ? W.B[k][lane] : 0.0;
        const double x1 = lane + 32 >= k ? W.B[k][lane + 32] : 0.0;
        const double nrm = sqrt(wsum(x0 * x0 + x1 * x1));
        if (!(nrm > 1e-7 * cn[k])) return false;
        const double bkk = W.B[k][k];
        const double alpha = bkk > 0.0 ? -nrm : nrm;
        __syncwarp();
        if (lane == 0) W.B[k][k] = bkk - alpha;
        __syncwarp();
        const double v0 = lane >= k ? W.B[k][lane] : 0.0;
        const double v1 = lane + 32 >= k ? W.B[k][lane + 32] : 0.0;
        const double beta = 2.0 / wsum(v0 * v0 + v1 * v1);
        if (lane == 0) {
            W.beta[k] = beta;
            W.rkk[k] = alpha;
        }
#pragma unroll
        for (int c = k + 1; c < M; c++) {
            const double dot = beta * wsum(v0 * W.B[c][lane] + v1 * W.B[c][lane + 32]);
            __syncwarp();
            if (lane >= k) W.B[c][lane] -= dot * v0;
            if (lane + 32 >= k) W.B[c][lane + 32] -= dot * v1;
            __syncwarp();
        }
    }
    __syncwarp();
    // z = R^-T e_1 (R_lk = B[k][l] for l < k, R_kk = rkk[k])
    double z[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        double a = k == 0 ? 1.0 : 0.0;
#pragma unroll
        for (int l = 0; l < k; l++) a -= W.B[k][l] * z[l];
        z[k] = a / W.rkk[k];
    }
    // y = H_0 ... H_{M-1} [z; 0], then N = sqrt(w) y
    double y0 = 0.0, y1 = 0.0;
#pragma unroll
    for (int k = 0; k < M; k++)
        if (lane == k) y0 = z[k];
#pragma unroll
    for (int k = M - 1; k >= 0; k--) {
        const double v0 = lane >= k ? W.B[k][lane] : 0.0;
        const double v1 = lane + 32 >= k ? W.B[k][lane + 32] : 0.0;
        const double dot = W.beta[k] * wsum(v0 * y0 + v1 * y1);
        y0 -= dot * v0;
        y1 -= dot * v1;
    }
    n0 = lane < cnt ? W.sw[lane] * y0 : 0.0;
    n1 = lane + 32 < cnt ? W.sw[lane + 32] * y1 : 0.0;
    __syncwarp();
    return true;
}

}  // namespace pcms
