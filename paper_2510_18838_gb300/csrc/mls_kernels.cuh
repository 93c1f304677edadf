// mls_kernels.cuh -- device code of the meshless MLS transfer (Sec. 3.2.1, Eq. 1).
//
// Per target t, the sources s_j with |s_j - t| < r (and phi > 0) are selected; with
// u_j = (s_j - t)/r, w_j = phi(|u_j|) and the graded-lex basis a(u) of degree k, the normal
// equations of Eq. 1 are G c = g with
//     G = sum_j w_j a(u_j) a(u_j)^T + lambda I,   g = sum_j w_j b_j a(u_j),
// and the transferred value is c_0 (a(0) = e_1). G's entries are moments
// M_p = sum_j w_j u_j^p over the monomials of degree <= 2k (15 instead of 21 entries in 2D
// quadratic, 35 instead of 55 in 3D quadratic), so a pair costs one multiply-add per
// moment. The cached operator stores N_j = w_j a(u_j)^T G^-1 e_1.
//
// Work split:
//   k_assemble  -- a group of G lanes per target walks the candidate cells (rows of
//                  contiguous cells in the counting-sorted source array), classifies
//                  candidates (FP32 hi/lo distance filter; pairs within 2^-16 of the
//                  radius are decided by the exact FP64 predicate), compacts the
//                  selected pairs through a shared-memory ring so the accumulation runs
//                  on full lanes, reduces the moments across the group and writes them.
//   k_solve     -- one thread per target: FP64 LDL^T of G with a pivot guard, then
//                  y = G^-1 e_1 (operator) or c_0 = e_1^T G^-1 g (one-shot transfer), and
//                  the routing of the mixed path's precision tiers (below).
//   k_shape     -- a group per target recomputes w_j a(u_j) and writes N_j.
#pragma once

#include <cmath>

#include "pcms_internal.cuh"

namespace pcms {

enum { MODE_COUNT = 0, MODE_MAP = 1, MODE_FUSED = 2 };

// How a group accumulates its moments.
//   ACC_PLAIN  one running sum per lane (FP32 on the mixed path, FP64 on the FP64 path),
//              lanes reduced in the same type.
//   ACC_BK     mixed path, blocked compensation: each lane adds BK_BLOCK selected pairs
//              into a plain FP32 block sum, then adds the block sum into a Kahan-compensated
//              FP32 total; lanes are reduced error-free (two-sum) and each moment is written
//              as an unevaluated FP32 pair (hi, lo). Everything stays on the FP32 pipe; the
//              summation error no longer grows with the neighbour count, so what is left is
//              the rounding of the individual terms, which averages out like 1/sqrt(n).
enum { ACC_PLAIN = 0, ACC_BK = 1 };
constexpr int BK_BLOCK = 4;
// Tier 1 of dense 2D one-shot targets (32 lanes per target, every lane adding its own
// candidate) uses blocks of BK_BLOCK_DENSE pairs: a quarter of the Kahan updates, calibrated
// with its own acceptance bound AMP_BK_DENSE (below). Tier 2, and 3D, keep BK_BLOCK.
constexpr int BK_BLOCK_DENSE = 16;
constexpr int DENSE_UNROLL = 4;   // candidates per lane per step of the dense form's walk

constexpr float MIX_BAND = 1.52587890625e-05f;   // 2^-16 relative band around r^2
constexpr int MAX_DOUBLINGS = 60;

// The radius after k doublings and what the kernels derive from it, computed once on the
// host. Kernels read these instead of deriving them in FP64: under register pressure the
// register allocator would otherwise recompute such values inside the candidate loop, and
// every FP64 instruction there costs 64 FP32 ones on this GPU.
struct RadiusLevels {
    double r[MAX_DOUBLINGS + 1];       // radius * 2^k
    double r2[MAX_DOUBLINGS + 1];      // r * r
    double inv_r[MAX_DOUBLINGS + 1];   // 1 / r
    float r2f[MAX_DOUBLINGS + 1];      // (float)(r * r)
    float inv_rf[MAX_DOUBLINGS + 1];   // (float)(1 / r)
    float rcell[MAX_DOUBLINGS + 1];    // the radius in cell units, (float)(r / h), at most 2^30
};

inline RadiusLevels make_radius_levels(double radius, double inv_h) {
    RadiusLevels L;
    for (int k = 0; k <= MAX_DOUBLINGS; k++) {
        const double r = std::ldexp(radius, k);
        L.r[k] = r;
        L.r2[k] = r * r;
        L.inv_r[k] = 1.0 / r;
        L.r2f[k] = (float)(r * r);
        L.inv_rf[k] = (float)(1.0 / r);
        L.rcell[k] = std::fmin((float)(r * inv_h), 1073741824.f);
    }
    return L;
}

struct AsmArgs {
    Grid g;
    int64_t ns, nt;
    const int32_t* cell_start;
    const double* sx64;   // [dim][ns] sorted sources
    const float4* hl0;    // mixed: sorted hi/lo
    const float2* hl1;
    const double* tx64;   // [dim][nt] sorted targets
    const float4* thl0;   // mixed: sorted targets' hi/lo (same layout as hl0/hl1)
    const float2* thl1;
    const int4* tcell;    // sorted targets' cell coordinates and positions in the cell
    const float4* tfrac;  // (point_cell)
    RadiusLevels lv;
    const int32_t* list;  // optional target list (length *n_list); moments then indexed by list position
    const int32_t* n_list;
    double radius;
    int weight;
    int need;
    const int32_t* kexp_in;  // starting doublings (MAP: exact; FUSED redo: start), or null
    int32_t* kexp_out;       // COUNT/FUSED
    int32_t* counts;
    int64_t* offsets;        // MAP: row starts (written in one-pass mode, read otherwise)
    int32_t* cols;           // MAP: column indices, or null (tiers 2/3 only need moments)
    // one-pass MAP (fixed radius): each group stages its target's columns in shared memory,
    // then reserves exact space with one atomic add on nnz_ctr; targets whose columns did
    // not fit the stage or the buffer (cols_cap) are listed in redo for a second walk
    int one_pass;
    unsigned long long* nnz_ctr;
    int64_t cols_cap;
    int32_t* redo;
    int32_t* n_redo;
    const void* field;       // FUSED: sorted field (float or double)
    void* mom;               // MAP/FUSED: [nt][NACCP] (float, float2 for ACC_BK, or double)
    const float4* basis;     // list mode (ACC_BK, or FP64): per list position (c_x, c_y, c_z, 1/s), or null
    // tier 1, blocked compensation: the sources' cell-sum pyramid (cell_pyramid: level j
    // starts at pyr_off[j]), from which a target whose radius grew, or whose ball reaches
    // past the grid, estimates its neighbours' weighted centroid and spread before it walks;
    // if the estimated centroid lies more than sqrt(recentre_min2) (offsets in units of the
    // radius) from the target, it is assembled in that re-centred basis. The basis used is
    // written to basis_out[t] (the identity when none). Null: target-centred.
    const float4* cpyr;
    int64_t pyr_off[PYR_MAX];
    int pyr_levels;
    float4* basis_out;
    float recentre_min2;
    unsigned* err;
};

// Precision tiers of the mixed path. The FP64 solve of a tier-1 system estimates how much
// the FP32 assembly error can move c_0 (amp, below) and hands sensitive targets on:
//   tier 1  plain FP32 (8-lane groups)      accepted if amp * (1 + sqrt(n / (3 G^2))) <= AMP_T1
//           blocked compensation (32 lanes) accepted if amp <= AMP_BK * sqrt(n)
//   tier 2  blocked compensation in a re-centred, re-scaled basis (lambda = 0; see below),
//           accepted if amp' <= AMP_BK * sqrt(n)
//   tier 3  FP64 assembly                   final (pivot guard TAU_FP64 only)
// A failed pivot guard in tier 1 or 2 also goes to tier 3. The bounds keep the estimated
// error of c_0 several times below 2e-5. They are calibrated on emulated FP32 arithmetic
// over the 2D Gaussian-mixture targets (field of unit size):
//   plain sums          err ~ amp * 6e-8 * (1 + sqrt(n / 3G^2));
//   blocked compensated err <= 3.4 * amp * 6e-8 / sqrt(n) (largest over 500 targets with
//                       up to 5e5 neighbours), so AMP_BK = 32 leaves a factor 3.
// A second emulation (600 uniform targets of the same case, up to 4.9e5 neighbours, lanes
// fed in stream order with unselected candidates as exact zeros) put the largest constant at
// 5.8 for blocks of 4 pairs and 8.3 for blocks of 16, the rounding of the terms alone at 4.9.
// Dense one-shot tier 1 (blocks of BK_BLOCK_DENSE = 16) therefore accepts amp <=
// AMP_BK_DENSE * sqrt(n) with AMP_BK_DENSE = 32 * 5.8 / 8.3 = 22: the same error bound as
// blocks of 4 under AMP_BK. In that sample 0.01% of the pairs belong to targets between the
// two bounds, which go to tier 2.
//
// Re-centred basis. Far targets (radius doubled until min_neighbors sources are inside)
// often see their neighbours on one side, at offsets u = (s - t)/r of size ~1 with a small
// spread. In the target-centred basis the normal equations are then badly scaled and amp is
// large, although the fit itself is not sensitive. At lambda = 0 the MLS value does not
// depend on the basis of the polynomial space, so tier 2 uses u' = (u - c)/s with c the
// weighted centroid and s the weighted spread of the tier-1 neighbours, and evaluates the
// fitted polynomial at u'_t = -c/s: G' y = a(u'_t), c_0 = y^T g'. (c, 1/s) are rounded to
// FP32 once and define the basis exactly for assembly, solve and operator rows.
//
// The FP64 path has the same sensitivity, 2^29 times smaller: FP64 normal equations give
// c_0 to about 15 * amp * 2^-53 (numpy on extrapolating 3D quadratic targets, amp up to
// 2e6). Its targets with amp > AMP_FP64 keep their target-centred status and values, and are
// assembled and solved once more in FP64 in the re-centred basis (the "refine" pass); if
// that solve passes its pivot guard its values replace the first ones. On extrapolating
// targets this cuts amp and the error by factors of 50 to 300.
constexpr double AMP_T1 = 64.0;
constexpr double AMP_BK = 32.0;
constexpr double AMP_BK_DENSE = 22.0;
constexpr double AMP_SHAPE = 32.0;   // operator rows above this are evaluated in FP64
constexpr double AMP_FP64 = 256.0;   // FP64 path: above this the error may pass 4e-13

struct SolveArgs {
    int64_t nt;
    const int32_t* list;
    const int32_t* n_list;
    const int32_t* counts;
    const void* mom;          // [nt or list][NACCP] (float or double)
    double lambda;
    double tau;               // pivot guard: d_k <= tau * G_kk fails
    int tier;                 // 1, 2 (mixed) or 3 (FP64)
    int group;                // lanes per target of the assembly (error model)
    int acc;                  // ACC_PLAIN or ACC_BK: how these moments were accumulated
    int recentre;             // tier 1 -> 2: hand on a re-centred basis (lambda = 0, degree >= 1)
    int refine64;             // FP64 path: list targets with amp > AMP_FP64 for the refine pass
    const float4* basis_in;   // basis of these moments: per list position (list mode), else
                              // per target (tier 1 with an estimated basis), or null
    int32_t* n_recentred;     // tier 1: targets solved in an estimated re-centred basis, or null
    int32_t* fb_list;         // mixed tiers: work items (wk) the refined FP32 solve declined,
    int32_t* n_fb;            // solved in FP64 by a second launch (k_solve<..., PASS 2>)
    // final FP64 solves (tier 3 not sent to the refine pass, tier 4) with amp / rho above
    // amp_qr (rho: the smallest LDL^T pivot ratio), and refine solves that fail their guard:
    // sorted targets for the Householder-QR pass (qr.cuh), or null
    int32_t* qr_list;
    int32_t* n_qr;
    float amp_qr;
    int32_t* list64;          // MAP: targets whose operator rows are FP64 (flag 2), or null
    int32_t* n64;
    float4* basis2;           // tier 1: basis for tier 2, per list2 position
    float4* rc;               // MAP: basis of the accepted tier-2 rows, per sorted target
    int32_t* list2;           // targets for tier 2 / tier 3
    int32_t* n2;
    int32_t* list3;
    int32_t* n3;
    double* y;                // MAP: [nt][m]
    float2* yf;               // mixed MAP: y as FP32 pairs {hi, lo} (y = hi + lo to ~2^-48)
    int8_t* flags;            // MAP: how to evaluate the operator row (k_shape)
    int8_t* status;           // MAP: sorted order; FUSED: caller order (via perm) or null
    const int32_t* perm_t;    // FUSED: sorted -> caller target index
    void* out;                // FUSED: caller-order output (float or double)
    int out_is_double;
};

struct ShapeArgs {
    Grid g;
    int64_t ns, nt;
    const double* sx64;
    const float4* hl0;
    const float2* hl1;
    const double* tx64;
    const float4* thl0;
    const float2* thl1;
    RadiusLevels lv;
    const int32_t* kexp;
    const int64_t* offsets;   // row starts
    const int32_t* counts;    // row lengths
    const int32_t* cols;
    const double* y;
    const float2* yf;   // mixed: y as FP32 pairs (written by the solve)
    const int8_t* flags;   // per target (mixed maps), or null: see k_shape
    const float4* rc;      // per target: re-centred basis of flag-3 rows
    double radius;
    int weight;
    void* vals;
    // k_shape<..., APPLY = true> (mixed): the rows are applied as they are evaluated instead of
    // stored: stage[t][f] = sum_i N_ti fs[col_i][f] for f < fp (fields in sorted source order,
    // fp = 1 or a multiple of 4 up to 16), NaN where status[t] is not OK
    const float* fs;
    int fp;
    const int8_t* status;
    float* stage;
};

// ------------------------------------------------------------------------------------
// weights (value only; selection is decided separately)
// ------------------------------------------------------------------------------------
template <typename T>
__host__ __device__ __forceinline__ T weight_value(int kind, T q) {
    const T one = T(1);
    switch (kind) {
    case PCMS_WENDLAND_C2: {
        T t = one - q;
        T t2 = t * t;
        return t2 * t2 * (T(4) * q + one);
    }
    case PCMS_GAUSSIAN: return exp(-(T(4) * q * q));
    case PCMS_C4: {
        T t = one - q;
        T t2 = t * t;
        T t6 = t2 * t2 * t2;
        T p = ((((T(5) * q + T(30)) * q + T(72)) * q + T(82)) * q + T(36)) * q + T(6);
        return p * t6;
    }
    case PCMS_MQ: return sqrt(one + T(4) * q * q);
    case PCMS_IMQ: return one / sqrt(one + T(4) * q * q);
    case PCMS_TPS: {
        T aq = T(2) * q;
        return aq == T(0) ? T(0) : aq * aq * log(aq);
    }
    case PCMS_CUBIC: {
        T aq = T(2) * q;
        return aq * aq * aq;
    }
    default: return one;  // CONST, NOOP
    }
}

// Exact selection, evaluated as the definition does: d2 < r*r and phi(sqrt(d2)/r) > 0 with
// IEEE sqrt and division. The sign of phi reduces to a test on q for every kind: Wendland
// and C4 are positive iff q < 1 (their factors cannot underflow for q < 1); Gaussian, MQ,
// IMQ, Const and No_Op are positive for every q < 1; TPS (2q)^2 ln(2q) iff 2q > 1; cubic
// (2q)^3 iff the product does not underflow to zero.
__device__ __forceinline__ bool select_exact(int kind, double d2, double r, double r2) {
    if (!(d2 < r2)) return false;
    double q = __ddiv_rn(__dsqrt_rn(d2), r);
    switch (kind) {
    case PCMS_WENDLAND_C2:
    case PCMS_C4: return q < 1.0;
    case PCMS_TPS: return __dmul_rn(2.0, q) > 1.0;
    case PCMS_CUBIC: {
        double aq = __dmul_rn(2.0, q);
        return __dmul_rn(__dmul_rn(aq, aq), aq) > 0.0;
    }
    default: return true;
    }
}

// FP64 selection with shortcuts that never change the decision
__device__ __forceinline__ bool select64(int kind, double d2, double r, double r2, double r2_in) {
    if (!(d2 < r2)) return false;
    if (kind == PCMS_TPS || kind == PCMS_CUBIC) return select_exact(kind, d2, r, r2);
    if (d2 < r2_in) return true;   // r2_in = r2 (1 - 2^-40): q < 1 certainly
    return select_exact(kind, d2, r, r2);
}

// FP32 classification: 1 inside, 0 outside, -1 decide exactly
__device__ __forceinline__ int classify32(int kind, float d2, float r2) {
    if (d2 > r2 * (1.0f + MIX_BAND)) return 0;
    const bool in_up = d2 < r2 * (1.0f - MIX_BAND);
    if (kind == PCMS_TPS) {
        const float q2 = 0.25f * r2;
        if (d2 < q2 * (1.0f - MIX_BAND)) return 0;
        if (d2 <= q2 * (1.0f + MIX_BAND)) return -1;
    } else if (kind == PCMS_CUBIC) {
        if (d2 < r2 * 9.094947e-13f) return -1;   // 2^-40
    }
    return in_up ? 1 : -1;
}

// exact FP64 squared distance, summed left to right without contraction
template <int DIM>
__device__ __forceinline__ double dist2_exact(const double* __restrict__ sx64, int64_t ns, int64_t j,
                                              const double* t) {
    double dx = __dsub_rn(sx64[j], t[0]);
    double dy = __dsub_rn(sx64[ns + j], t[1]);
    double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (DIM == 3) {
        double dz = __dsub_rn(sx64[2 * ns + j], t[2]);
        d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
    }
    return d2;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// source index carried through the queue's payload slot, bit-exact
__device__ __forceinline__ float pack_index(int j, float) { return __int_as_float(j); }
__device__ __forceinline__ double pack_index(int j, double) { return (double)j; }
__device__ __forceinline__ int unpack_index(float v) { return __float_as_int(v); }
__device__ __forceinline__ int unpack_index(double v) { return (int)v; }

template <typename T> struct QEntry;
template <> struct QEntry<float> { using type = float4; };
template <> struct QEntry<double> { using type = double4_32a; };

template <typename T>
__device__ __forceinline__ typename QEntry<T>::type make_entry(T a, T b, T c, T d);
template <>
__device__ __forceinline__ float4 make_entry<float>(float a, float b, float c, float d) {
    return make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ double4_32a make_entry<double>(double a, double b, double c, double d) {
    return make_double4_32a(a, b, c, d);
}

// accumulate one selected pair: dx (target-relative offsets), payload b (field value)
// s += x with Kahan's compensation c (the true running sum is s - c)
template <typename T>
__host__ __device__ __forceinline__ void kahan_add(T& s, T& c, T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// Error-free sum of two FP32 values (Knuth's TwoSum): s + e == a + b exactly.
__host__ __device__ __forceinline__ void two_sum32(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Offsets u = dx / r of one selected pair in the assembly basis: target-centred, or with
// bc = {c_x, c_y, c_z, 1/s} the re-centred basis u' = (u - c) / s.
template <int DIM, typename T>
__host__ __device__ __forceinline__ void basis_offsets(const T* dx, T inv_r, const T* bc, T* u) {
    u[0] = dx[0] * inv_r;
    u[1] = dx[1] * inv_r;
    u[2] = DIM == 3 ? dx[2] * inv_r : T(0);
    if (bc) {
#pragma unroll
        for (int d = 0; d < DIM; d++) u[d] = (u[d] - bc[d]) * bc[3];
    }
}

// Pairing of the moment terms w u^p (graded order, p >= 1) for two-lane FP32 arithmetic. Each
// term is its parent (the monomial with its first positive exponent lowered) times the offset
// of that variable, as in the scalar chain. Degree by degree, a term p joins the term q of the
// same variable whose parent is the partner of p's parent: the pair is then one packed
// product (parent pair times the offset in both lanes). The terms left over in a degree are
// paired in order; their products stay scalar but their sums, and the next degree's products
// of their children, are packed. partner[p] = -1 for a term left alone; first[p] marks the
// lane-0 term of a pair, packed[p] a pair whose product is packed.
template <int DIM, int MDEG>
struct PairPlan {
    static constexpr int N = mono_count(DIM, MDEG);
    int partner[N];
    bool first[N];
    bool packed[N];
};
template <int DIM, int MDEG>
__host__ __device__ constexpr PairPlan<DIM, MDEG> make_pair_plan() {
    PairPlan<DIM, MDEG> P{};
    for (int p = 0; p < PairPlan<DIM, MDEG>::N; ++p) {
        P.partner[p] = -1;
        P.first[p] = false;
        P.packed[p] = false;
    }
    for (int d = 1; d <= MDEG; ++d) {
        const int lo = mono_count(DIM, d - 1), hi = mono_count(DIM, d);
        for (int p = lo; p < hi; ++p) {
            if (P.partner[p] >= 0) continue;
            const int a = mono_parent(DIM, p), v = mono_var(DIM, p);
            if (P.partner[a] < 0 || !P.first[a]) continue;
            const Exp3 eb = mono_exp(DIM, P.partner[a]);
            int e[3] = {eb.e[0], eb.e[1], eb.e[2]};
            e[v] += 1;
            const int q = mono_index(DIM, e[0], e[1], e[2]);
            if (q < lo || q >= hi || q == p || P.partner[q] >= 0 || mono_var(DIM, q) != v) continue;
            P.partner[p] = q;
            P.partner[q] = p;
            P.first[p] = true;
            P.packed[p] = true;
        }
        int s = -1;
        for (int p = lo; p < hi; ++p) {
            if (P.partner[p] >= 0) continue;
            if (s < 0) {
                s = p;
            } else {
                P.partner[s] = p;
                P.partner[p] = s;
                P.first[s] = true;
                s = -1;
            }
        }
    }
    return P;
}
template <int DIM, int MDEG>
struct PairPlanOf {
    static constexpr PairPlan<DIM, MDEG> v = make_pair_plan<DIM, MDEG>();
};

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// The FP32 moment chain and its sums on two-lane FP32 instructions (multiply, add and fused
// multiply-add on a pair of FP32 values, one instruction per pair): every term is the same
// product of its parent and one offset as in the scalar chain, so only the instruction count
// changes (2D quadratic: 24 -> 16 per pair, 3D quadratic: 54 -> 33). Terms of the top degree
// have no children and go straight into their sums (fused multiply-add). In fused mode the
// right-hand side w b u^p (degree <= k) takes the same pairs.
template <int DIM, int DEG, int MODE, int N>
__device__ __forceinline__ void chain_packed(float (&acc)[N], float w, const float* u, float b) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int TOP = mono_count(DIM, 2 * DEG - 1);   // first term of the top degree
    using PP = PairPlanOf<DIM, 2 * DEG>;
    float wm[NM];
    wm[0] = w;
    acc[0] += w;
    sfor<NM - 1>([&](auto I) {
        constexpr int p = decltype(I)::value + 1;
        constexpr int q = PP::v.partner[p];
        constexpr int pa = mono_parent(DIM, p);
        constexpr int va = mono_var(DIM, p);
        constexpr bool top = p >= TOP;
        if constexpr (q < 0) {
            if constexpr (top) {
                acc[p] = fmaf(wm[pa], u[va], acc[p]);
            } else {
                wm[p] = wm[pa] * u[va];
                acc[p] += wm[p];
            }
        } else if constexpr (PP::v.first[p]) {
            constexpr int pb = mono_parent(DIM, q);
            constexpr int vb = mono_var(DIM, q);
            float2 s2 = make_float2(acc[p], acc[q]);
            if constexpr (PP::v.packed[p]) {
                const float2 par2 = make_float2(wm[pa], wm[pb]);
                const float2 uu = make_float2(u[va], u[va]);
                if constexpr (top) {
                    s2 = __ffma2_rn(par2, uu, s2);
                } else {
                    const float2 m2 = __fmul2_rn(par2, uu);
                    wm[p] = m2.x;
                    wm[q] = m2.y;
                    s2 = __fadd2_rn(s2, m2);
                }
            } else if constexpr (top) {
                s2.x = fmaf(wm[pa], u[va], s2.x);
                s2.y = fmaf(wm[pb], u[vb], s2.y);
            } else {
                wm[p] = wm[pa] * u[va];
                wm[q] = wm[pb] * u[vb];
                s2 = __fadd2_rn(s2, make_float2(wm[p], wm[q]));
            }
            acc[p] = s2.x;
            acc[q] = s2.y;
        }
    });
    if constexpr (MODE == MODE_FUSED) {
        acc[NM] = fmaf(w, b, acc[NM]);
        const float2 bb = make_float2(b, b);
        sfor<M - 1>([&](auto I) {
            constexpr int p = decltype(I)::value + 1;
            constexpr int q = PP::v.partner[p];
            if constexpr (q < 0) {
                acc[NM + p] = fmaf(wm[p], b, acc[NM + p]);
            } else if constexpr (PP::v.first[p]) {
                const float2 s2 = __ffma2_rn(make_float2(wm[p], wm[q]), bb,
                                             make_float2(acc[NM + p], acc[NM + q]));
                acc[NM + p] = s2.x;
                acc[NM + q] = s2.y;
            }
        });
    }
}
#endif

// Adds one selected pair to the running sums: moments w u^p of degree <= 2k, and in fused
// mode the right-hand side w b u^p of degree <= k. dx = target-relative offsets (the weight
// is always a function of |dx| / r), b = field value, bc = re-centred basis or null.
// WK >= 0 fixes the weight kind at compile time (the runtime kind is then ignored).
template <int DIM, int DEG, int MODE, typename T, int NACC, int WK = -1>
__host__ __device__ __forceinline__ void accumulate(T (&acc)[NACC > 0 ? NACC : 1], const T* dx,
                                                    T b, int kind, T inv_r, const T* bc,
                                                    bool selected = true) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    T d2 = dx[0] * dx[0] + dx[1] * dx[1];
    if (DIM == 3) d2 += dx[2] * dx[2];
    T q;
#ifdef __CUDA_ARCH__
    if constexpr (std::is_same<T, float>::value) q = sqrt_approx(d2) * inv_r;
    else q = sqrt(d2) * inv_r;
#else
    q = sqrt(d2) * inv_r;
#endif
    T w = weight_value<T>(WK >= 0 ? WK : kind, q);
    if (!selected) w = T(0);   // adds exact zeros: an unselected candidate leaves the sums as they are
    T u[3];
    basis_offsets<DIM, T>(dx, inv_r, bc, u);
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    if constexpr (std::is_same<T, float>::value && DEG >= 1) {
        chain_packed<DIM, DEG, MODE>(acc, w, u, b);
    } else
#endif
    {
        T wm[NM];
        wm[0] = w;
        acc[0] += w;
        sfor<NM - 1>([&](auto I) {
            constexpr int p = decltype(I)::value + 1;
            constexpr int par = mono_parent(DIM, p);
            constexpr int v = mono_var(DIM, p);
            wm[p] = wm[par] * u[v];
            acc[p] += wm[p];
        });
        if constexpr (MODE == MODE_FUSED) {
            // the basis monomials come first in the graded order, so w u^p of degree <= k is
            // already among the moment terms: one multiply-add per right-hand-side entry
            sfor<M>([&](auto I) {
                constexpr int p = decltype(I)::value;
                acc[NM + p] += wm[p] * b;
            });
        }
    }
}

// Blocked compensation: the block sums acc are added into the Kahan totals (sum, cmp) and
// cleared.
template <int NACC>
__host__ __device__ __forceinline__ void bk_flush(float (&acc)[NACC], float (&sum)[NACC],
                                                  float (&cmp)[NACC]) {
#pragma unroll
    for (int i = 0; i < NACC; i++) {
        kahan_add(sum[i], cmp[i], acc[i]);
        acc[i] = 0.f;
    }
}

// A lane's Kahan totals of blocked compensation: (sum, cmp) per running sum, the true total
// being sum - cmp. Kept in registers, or (SMEM) in the block's shared memory at
// base[i * 256] (one float2 per sum, 256 threads per block), which frees 2 NA registers
// for the dense one-shot form, whose block flushes are rare.
template <int NA, bool SMEM>
struct KahanTotals {
    float sum[NA], cmp[NA];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int i = 0; i < NA; i++) {
            sum[i] = 0.f;
            cmp[i] = 0.f;
        }
    }
    __device__ __forceinline__ void flush(float (&acc)[NA]) { bk_flush<NA>(acc, sum, cmp); }
    __device__ __forceinline__ float2 pair(int i) const { return make_float2(sum[i], -cmp[i]); }
};
template <int NA>
struct KahanTotals<NA, true> {
    float2* base;
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int i = 0; i < NA; i++) base[i * 256] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void flush(float (&acc)[NA]) {
#pragma unroll
        for (int i = 0; i < NA; i++) {
            float2 v = base[i * 256];
            kahan_add(v.x, v.y, acc[i]);
            base[i * 256] = v;
            acc[i] = 0.f;
        }
    }
    __device__ __forceinline__ float2 pair(int i) const {
        const float2 v = base[i * 256];
        return make_float2(v.x, -v.y);
    }
};

// ------------------------------------------------------------------------------------
// k_assemble
// ------------------------------------------------------------------------------------
// FP32 hi/lo coordinates of point i (relative to the grid origin) in the sorted hi/lo layout
template <int DIM>
__device__ __forceinline__ void load_hilo(const float4* h0, const float2* h1, int64_t i,
                                          float* hi, float* lo) {
    const float4 a = h0[i];
    if (DIM == 2) {
        hi[0] = a.x;
        hi[1] = a.y;
        lo[0] = a.z;
        lo[1] = a.w;
    } else {
        const float2 b = h1[i];
        hi[0] = a.x;
        hi[1] = a.y;
        hi[2] = a.z;
        lo[0] = a.w;
        lo[1] = b.x;
        lo[2] = b.y;
    }
}

// One candidate's data as the assembly walk loads it a step ahead: the hi/lo FP32
// coordinates (mixed) or the FP64 coordinates, and in fused mode the field value.
template <bool MIXED, int DIM, typename FT, bool LOADF>
struct Cand {
    float4 h0;
    float2 h1;
    double x[3];
    FT f;
    __device__ __forceinline__ void load(const AsmArgs& A, int j) {
        if constexpr (MIXED) {
            h0 = A.hl0[j];
            if constexpr (DIM == 3) h1 = A.hl1[j];
        } else {
            x[0] = A.sx64[j];
            x[1] = A.sx64[A.ns + j];
            if constexpr (DIM == 3) x[2] = A.sx64[2 * A.ns + j];
        }
        if constexpr (LOADF) f = ((const FT*)A.field)[j];
    }
};

// Stored moment type: T for ACC_PLAIN, an unevaluated FP32 pair for ACC_BK.
template <typename T, int ACC>
using MomT = typename std::conditional<ACC == ACC_BK, float2, T>::type;

// Two blocks per SM (at most 128 registers) except: the blocked 3D quadratic form, whose
// three accumulator sets of 35-45 moments would spill heavily at that size (one block); and
// three blocks (80 registers) for plain FP32 sums of at most 15 moments (degree <= 1, or 2D)
// and for the dense 2D one-shot form (its Kahan totals in shared memory): the walk is
// latency-bound, and the extra warps cut the serving stream's assembly time by 9% and the
// dense 2D transfer's by 2%, despite a few dozen bytes of spills.
template <int DIM, int DEG, int ACC, bool MIXED, int MODE, int G>
constexpr int asm_min_blocks() {
    return (ACC == ACC_BK && DIM == 3 && DEG == 2)
               ? 1
               : ((MIXED && ACC == ACC_PLAIN && (DEG <= 1 || DIM == 2)) ||
                          (ACC == ACC_BK && MODE == MODE_FUSED && G == 32 && DIM == 2)
                      ? 3
                      : 2);
}

// Candidate row rho of a target (cell (ct) and position in it (fr), cell units): the cells
// (dz, dy) in row-major order over [z0, z0 + nz) x [y0, y0 + ny), trimmed in x to the chord of
// the ball of radius RR (which includes the margin mg; y and z units, g.xs x cells per unit).
// Returns false for an empty row, else the row's first cell index and its x range [x0, x1],
// clamped to the grid.
template <int DIM>
__device__ __forceinline__ bool row_chord(const Grid& g, const long long* ct, const float* fr,
                                          float RR, float mg, long long y0, long long z0,
                                          long long ny, long long rho, int64_t& rowbase,
                                          long long& x0, long long& x1) {
    long long dz = 0, dy = y0 + rho;
    if (DIM == 3) {   // row counts are bounded by the grid's <= 2^24 cells
        const int q = (int)rho / (int)ny;
        dz = z0 + q;
        dy = y0 + ((int)rho - q * (int)ny);
    }
    float ez = 0.f;
    if (DIM == 3) {
        ez = fmaxf(fmaxf((float)dz - fr[2], fr[2] - (float)dz - 1.f), 0.f);
        ez = fmaxf(ez - mg, 0.f);
    }
    float ey = fmaxf(fmaxf((float)dy - fr[1], fr[1] - (float)dy - 1.f), 0.f);
    ey = fmaxf(ey - mg, 0.f);
    const float remz = RR * RR - ez * ez;
    const float rem = remz - ey * ey;
    if (!(remz > 0.f && rem > 0.f)) return false;
    const float hx = (sqrtf(rem) + mg) * (float)g.xs;
    x0 = max((long long)__float2int_rd(fr[0] - hx) + ct[0], 0LL);
    x1 = min((long long)__float2int_rd(fr[0] + hx) + ct[0], (long long)g.n[0] - 1);
    if (x0 > x1) return false;
    rowbase = ((ct[2] + dz) * g.n[1] + (ct[1] + dy)) * (int64_t)g.n[0];
    return true;
}

// The target's re-centred basis estimated from the sources' cell-sum pyramid (all G lanes of
// the group call this together). At radius level k it reads level j = min(k, top), whose
// entries span 2^j cells per axis, so the ball (3 or 2 cells per radius at k = 0) covers a
// few entries per axis at every k: the entries of the ball's bounding box, split over the
// lanes. Each entry contributes its count times the weight at its sources' mean position,
// u = (mean - t) / r. c = the weighted mean of u; s^2 = the weighted variance per axis plus
// that of a uniform entry, (2^j / cells per radius)^2 / 12. Returns (c, 1/s) rounded to
// FP32, or the identity (0, 0, 0, 1) when |c|^2 <= recentre_min2 or the estimate is
// degenerate: only markedly one-sided neighbourhoods change basis.
template <int DIM, int G>
__device__ __forceinline__ float4 estimate_basis(const AsmArgs& A, const long long* ct,
                                                 const float* fr, const float* thi, float RR,
                                                 float R0, float inv_r, int k, int gl,
                                                 unsigned gmask) {
    const float4 ident = make_float4(0.f, 0.f, 0.f, 1.f);
    const int j = min(k, A.pyr_levels - 1);
    const float4* lev = A.cpyr + A.pyr_off[j];
    int lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1}, nb[3] = {1, 1, 1};
    bool empty = false;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        // the pyramid is over h-wide cells: x positions in x cells are divided by xs
        const long long nd = d == 0 ? A.g.ncoarse_x() : A.g.n[d];
        nb[d] = (int)((nd + (1LL << j) - 1) >> j);
        const float p = d == 0 ? ((float)ct[0] + fr[0]) / (float)A.g.xs : (float)ct[d] + fr[d];
        // floor(x / 2^j) of the floored cell coordinates (arithmetic shifts floor negatives)
        const int a = max(__float2int_rd(p - RR) >> j, 0);
        const int b = min(__float2int_rd(p + RR) >> j, nb[d] - 1);
        empty = empty || a > b;
        lo[d] = a;
        ext[d] = b - a + 1;
    }
    if (empty) return ident;
    float s0 = 0.f, s1[3] = {0.f, 0.f, 0.f}, s2 = 0.f;
    const int total = ext[0] * ext[1] * ext[2];
    for (int i = gl; i < total; i += G) {
        const int ix = i % ext[0], r = i / ext[0], iy = r % ext[1], iz = r / ext[1];
        const int64_t idx =
            ((int64_t)(lo[2] + iz) * nb[1] + (lo[1] + iy)) * (int64_t)nb[0] + (lo[0] + ix);
        const float4 cs = lev[idx];
        if (!(cs.w > 0.f)) continue;
        const float inv_n = 1.f / cs.w;
        float u[3] = {(cs.x * inv_n - thi[0]) * inv_r, (cs.y * inv_n - thi[1]) * inv_r,
                      DIM == 3 ? (cs.z * inv_n - thi[2]) * inv_r : 0.f};
        const float q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        if (!(q2 < 1.f)) continue;
        const float w = cs.w * weight_value<float>(A.weight, sqrtf(q2));
        s0 += w;
#pragma unroll
        for (int d = 0; d < DIM; d++) s1[d] += w * u[d];
        s2 += w * q2;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(gmask, s0, o);
#pragma unroll
        for (int d = 0; d < DIM; d++) s1[d] += __shfl_xor_sync(gmask, s1[d], o);
        s2 += __shfl_xor_sync(gmask, s2, o);
    }
    if (!(s0 > 0.f)) return ident;
    float c[3] = {0.f, 0.f, 0.f}, cc = 0.f;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        c[d] = s1[d] / s0;
        cc += c[d] * c[d];
    }
    if (!(cc > A.recentre_min2)) return ident;
    const float e = (float)(1 << j) / R0;
    const float var = (s2 / s0 - cc) / (float)DIM + e * e / 12.f;
    if (!(var > 1e-12f)) return ident;
    return make_float4(c[0], c[1], c[2], 1.f / sqrtf(var));
}

template <int DIM, int DEG, bool MIXED, int MODE, int G, typename FT, int ACC = ACC_PLAIN>
__global__ void __launch_bounds__(256, asm_min_blocks<DIM, DEG, ACC, MIXED, MODE, G>()) k_assemble(AsmArgs A) {
    static_assert(ACC == ACC_PLAIN || (MIXED && MODE != MODE_COUNT), "blocked compensation: mixed moments only");
    using T = typename std::conditional<MIXED, float, double>::type;
    using MT = MomT<T, ACC>;
    using QE = typename QEntry<T>::type;
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NACC = MODE == MODE_FUSED ? NM + M : (MODE == MODE_MAP ? NM : 0);
    constexpr int NACCP = round_up4(NACC > 0 ? NACC : 1);
    constexpr int GPW = 32 / G;
    constexpr int QCAP = 2 * G;
    __shared__ QE qbuf[8][64];
    // Rows are set up RB = G * RPL at a time, RPL consecutive rows per lane: for the 8-lane 3D
    // walks (25 rows at the start radius) one batch instead of four, so the cell-start loads
    // of all rows are in flight together.
    constexpr int RPL = (DIM == 3 && G == 8) ? 4 : 1;
    constexpr int RB = G * RPL;
    __shared__ int rowa_s[8][32 * RPL], rowe_s[8][32 * RPL];   // per group: RB rows' source
                                                                // start, stream end

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gi = lane / G, gl = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
    const unsigned lt = (1u << lane) - 1u;
    QE* q = &qbuf[wib][gi * QCAP];
    int* rA = &rowa_s[wib][gi * RB];
    int* rE = &rowe_s[wib][gi * RB];
    // one-pass MAP: staged column indices, STG per group (24 KB per block)
    constexpr int STG = MODE == MODE_MAP ? (G == 32 ? 768 : 192) : 1;
    __shared__ int32_t stg_s[MODE == MODE_MAP ? 8 * GPW * STG : 1];
    int32_t* stg = &stg_s[MODE == MODE_MAP ? (wib * GPW + gi) * STG : 0];
    using CandT = Cand<MIXED, DIM, FT, MODE == MODE_FUSED>;
    // Dense one-shot targets (warp per target, blocked compensation): about 3 in 4 candidates
    // are selected, so every lane accumulates its own candidate with the weight zeroed when it
    // is not selected, instead of compacting selected pairs through the shared-memory ring.
    constexpr bool PRED = MODE == MODE_FUSED && ACC == ACC_BK && G == 32;
    const int bk_block = (PRED && DIM == 2 && !A.list) ? BK_BLOCK_DENSE : BK_BLOCK;
    // the dense form's Kahan totals live in shared memory where they fit the static limit
    constexpr int NA = NACC > 0 ? NACC : 1;
    constexpr bool SMEM_TOT = PRED && NA * 256 * 8 <= 44 * 1024;
    __shared__ float2 tot_s[SMEM_TOT ? NA * 256 : 1];

    const int64_t ngroups = (int64_t)gridDim.x * (blockDim.x >> 5) * GPW;
    const int64_t gid = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GPW + gi;
    const int64_t nwork = A.list ? (int64_t)(*A.n_list) : A.nt;
    const Grid& g = A.g;

    for (int64_t wk = gid; wk < nwork; wk += ngroups) {
        const int64_t t = A.list ? (int64_t)A.list[wk] : wk;
        // The target's cell and position in it were computed once when the targets were
        // sorted; its FP64 coordinates are only read by the FP64 path (and, on the mixed
        // path, by the rare exact decision), which keeps FP64 work out of the target set-up
        // that all G lanes of the group repeat.
        double tx[3] = {0.0, 0.0, 0.0};
        long long ct[3] = {0, 0, 0};
        float fr[3] = {0.f, 0.f, 0.f};
        {
            const int4 c4 = A.tcell[t];
            const float4 f4 = A.tfrac[t];
            ct[0] = c4.x;
            ct[1] = c4.y;
            ct[2] = c4.z;
            fr[0] = f4.x;
            fr[1] = f4.y;
            fr[2] = f4.z;
        }
        if constexpr (!MIXED) {
#pragma unroll
            for (int d = 0; d < DIM; d++) tx[d] = A.tx64[d * A.nt + t];
        }
        float thi[3] = {0.f, 0.f, 0.f}, tlo[3] = {0.f, 0.f, 0.f};
        if constexpr (MIXED) load_hilo<DIM>(A.thl0, A.thl1, t, thi, tlo);
        int k = A.kexp_in ? A.kexp_in[t] : 0;
        int cnt = 0;
        int64_t row_off = 0, row_len = 0;
        const bool one_pass = MODE == MODE_MAP && A.one_pass;
        if (MODE == MODE_MAP && !one_pass && A.cols) {   // a previous pass fixed the row
            row_off = A.offsets[t];
            row_len = A.counts[t];
        }
        // re-centred basis (blocked tier 2, FP64 refine pass)
        T bcv[4] = {T(0), T(0), T(0), T(1)};
        const T* bc = nullptr;
        if constexpr (ACC == ACC_BK || !MIXED) {
            if (A.basis) {
                const float4 bb = A.basis[wk];
                bcv[0] = bb.x;
                bcv[1] = bb.y;
                bcv[2] = bb.z;
                bcv[3] = bb.w;
                bc = bcv;
            }
        }
        constexpr int NB = ACC == ACC_BK ? NA : 1;   // Kahan totals (blocked compensation)
        T acc[NA];
        KahanTotals<NB, SMEM_TOT> tot;
        if constexpr (SMEM_TOT) tot.base = &tot_s[threadIdx.x];
        int pops = 0;
        for (;;) {
            const double r = A.lv.r[k];
            const double r2 = A.lv.r2[k];
            const double r2_in = r2 * (1.0 - 9.094947017729282e-13);
            const float r2f = A.lv.r2f[k];
            T inv_r;
            if constexpr (MIXED) inv_r = A.lv.inv_rf[k];
            else inv_r = A.lv.inv_r[k];
            // Candidate rows: cells (y, z) whose slab comes within r of the target, each
            // trimmed in x to the ball's chord. Computed in cell units in FP32 with a margin
            // m far above the FP32 error, so the rows and chords only ever over-cover. The
            // floors are 32-bit conversions rounding down (|argument| < 2^31 since the radius
            // is capped at 2^30 cells): a 64-bit conversion would run on the FP64 pipe.
            const float R0 = A.lv.rcell[k];
            const float mg = 1e-3f + R0 * 1e-6f;
            const float RR = R0 + mg;
            long long z0 = 0, z1 = 0;
            if (DIM == 3) {
                z0 = max((long long)__float2int_rd(fr[2] - RR), -ct[2]);
                z1 = min((long long)__float2int_rd(fr[2] + RR), (long long)g.n[2] - 1 - ct[2]);
            }
            const long long y0 = max((long long)__float2int_rd(fr[1] - RR), -ct[1]);
            const long long y1 = min((long long)__float2int_rd(fr[1] + RR), (long long)g.n[1] - 1 - ct[1]);
            const long long ny = y1 >= y0 ? y1 - y0 + 1 : 0;
            const long long nrows = ny * (DIM == 3 ? (z1 >= z0 ? z1 - z0 + 1 : 0) : 1);
            // (before the sums are cleared, so that they are not live across it)
            if constexpr (MIXED && ACC == ACC_BK && MODE != MODE_COUNT) {
                // tier 1: this level's estimated basis, for the targets whose neighbourhood
                // can be one-sided: a grown radius, or a ball that reaches past the grid
                bool want = k > 0;
#pragma unroll
                for (int d = 0; d < DIM; d++) {
                    const float p = (float)ct[d] + fr[d];
                    const float rd = d == 0 ? RR * (float)g.xs : RR;
                    want = want || p - rd < 0.f || p + rd > (float)g.n[d];
                }
                if (A.cpyr && !A.list) {
                    const float4 eb =
                        want ? estimate_basis<DIM, G>(A, ct, fr, thi, RR, R0, inv_r, k, gl, gmask)
                             : make_float4(0.f, 0.f, 0.f, 1.f);
                    bcv[0] = eb.x;
                    bcv[1] = eb.y;
                    bcv[2] = eb.z;
                    bcv[3] = eb.w;
                    const bool ident = eb.x == 0.f && eb.y == 0.f && eb.z == 0.f && eb.w == 1.f;
                    bc = ident ? nullptr : bcv;
                }
            }
#pragma unroll
            for (int i = 0; i < NA; i++) acc[i] = T(0);
            if constexpr (ACC == ACC_BK) tot.clear();
            pops = 0;
            cnt = 0;
            int qn = 0, head = 0;
            int64_t written = 0;
            // The rows are taken G at a time: each lane sets up one row (its chord and the
            // range [a, a + len) of cell-sorted sources it covers), a prefix sum over the
            // group lays those ranges end to end, and the group streams the concatenated
            // candidates G per step, so steps are full across row ends. The loads of the
            // next step are issued before the current one is classified.
            for (long long row0 = 0; row0 < nrows; row0 += RB) {
                int64_t cs0[RPL], cs1[RPL];   // cell-start indices of each row's x range
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
                    const int v = __shfl_up_sync(gmask, incl, o, G);
                    if (gl >= o) incl += v;
                }
                const int total = __shfl_sync(gmask, incl, G - 1, G);
                int e = incl - lsum;
#pragma unroll
                for (int i = 0; i < RPL; i++) {
                    e += rl[i];
                    rA[gl * RPL + i] = ra[i];
                    rE[gl * RPL + i] = e;
                }
                __syncwarp(gmask);
                if constexpr (PRED) {
                    // Each lane keeps its own cursor into the batch of rows: its stream position
                    // advances by G per step, and within a row the source index does too,
                    // so the row table is read only where a lane crosses into a later row.
                    // Steps are taken DU at a time while DU full steps remain (one row check,
                    // one check for FP32-undecided pairs and one block-flush check per DU
                    // candidates of a lane), then one at a time. Each lane counts its own
                    // selected pairs; the group's count is reduced after the walk.
                    auto stream = [&](auto wkc) {
                        constexpr int WK = decltype(wkc)::value;
                        constexpr int DU = DENSE_UNROLL;
                        int rcur = 0, pos = gl, pend = 0, jc = 0;   // jc: source at pos
                        if (pos < total) {
                            while (rE[rcur] <= pos) ++rcur;
                            pend = rE[rcur];
                            jc = rA[rcur] + pos - (rcur ? rE[rcur - 1] : 0);
                        }
                        // move the cursor one step (pos < total before the step)
                        auto step = [&]() {
                            pos += G;
                            if (pos < pend) {
                                jc += G;
                            } else if (pos < total) {   // the loop moves rcur at least once
                                while (rE[rcur] <= pos) ++rcur;
                                pend = rE[rcur];
                                jc = rA[rcur] + pos - rE[rcur - 1];
                            }
                        };
                        // offsets and FP32 classification of one candidate: 1 in, 0 out,
                        // -1 undecided in FP32
                        auto classify = [&](const CandT& c, T* dx) -> int {
                            float ddx, ddy, ddz = 0.f;
                            if (DIM == 2) {
                                ddx = (c.h0.x - thi[0]) + (c.h0.z - tlo[0]);
                                ddy = (c.h0.y - thi[1]) + (c.h0.w - tlo[1]);
                            } else {
                                ddx = (c.h0.x - thi[0]) + (c.h0.w - tlo[0]);
                                ddy = (c.h0.y - thi[1]) + (c.h1.x - tlo[1]);
                                ddz = (c.h0.z - thi[2]) + (c.h1.y - tlo[2]);
                            }
                            float d2f = ddx * ddx + ddy * ddy;
                            if (DIM == 3) d2f += ddz * ddz;
                            dx[0] = ddx;
                            dx[1] = ddy;
                            dx[2] = ddz;
                            if constexpr (WK == PCMS_WENDLAND_C2)   // classify32 for this kind
                                return d2f > r2f * (1.0f + MIX_BAND)
                                           ? 0
                                           : (d2f < r2f * (1.0f - MIX_BAND) ? 1 : -1);
                            else
                                return classify32(A.weight, d2f, r2f);
                        };
                        auto exact = [&](int j) -> bool {
                            double te[3] = {0.0, 0.0, 0.0};
#pragma unroll
                            for (int d = 0; d < DIM; d++) te[d] = A.tx64[d * A.nt + t];
                            return select_exact(A.weight, dist2_exact<DIM>(A.sx64, A.ns, j, te), r,
                                                r2) != 0;
                        };
                        int p0 = 0;
                        for (; p0 + DU * G <= total; p0 += DU * G) {
                            int jj[DU];
                            CandT cc[DU];
#pragma unroll
                            for (int u = 0; u < DU; u++) {
                                jj[u] = jc;
                                cc[u].load(A, jc);
                                if (u + 1 < DU) step();
                            }
                            step();
                            T dx[DU][3];
                            int cl[DU];
                            bool und = false;
#pragma unroll
                            for (int u = 0; u < DU; u++) {
                                cl[u] = classify(cc[u], dx[u]);
                                und = und || cl[u] < 0;
                            }
                            if (und) {
#pragma unroll
                                for (int u = 0; u < DU; u++)
                                    if (cl[u] < 0) cl[u] = exact(jj[u]) ? 1 : 0;
                            }
#pragma unroll
                            for (int u = 0; u < DU; u++) {
                                cnt += cl[u];
                                accumulate<DIM, DEG, MODE, T, NACC, WK>(acc, dx[u], (T)cc[u].f,
                                                                        A.weight, inv_r, bc,
                                                                        cl[u] != 0);
                            }
                            pops += DU;
                            if (pops >= bk_block) {
                                tot.flush(acc);
                                pops = 0;
                            }
                        }
                        for (; p0 < total; p0 += G) {
                            const bool v = pos < total;
                            const int j = jc;
                            CandT c;
                            if (v) {
                                c.load(A, j);
                                step();
                            }
                            T dx[3] = {T(0), T(0), T(0)};
                            int cl = 0;
                            if (v) {
                                cl = classify(c, dx);
                                if (cl < 0) cl = exact(j) ? 1 : 0;
                            }
                            cnt += cl;
                            accumulate<DIM, DEG, MODE, T, NACC, WK>(acc, dx, v ? (T)c.f : T(0),
                                                                    A.weight, inv_r, bc, cl != 0);
                            if (++pops >= bk_block) {
                                tot.flush(acc);
                                pops = 0;
                            }
                        }
                    };
                    if (A.weight == PCMS_WENDLAND_C2)
                        stream(std::integral_constant<int, PCMS_WENDLAND_C2>{});
                    else
                        stream(std::integral_constant<int, -1>{});
                    __syncwarp(gmask);   // the row table is rewritten by the next RB rows
                    continue;
                }
                // Selected pairs are compacted through the group's ring so that accumulation
                // runs on full lanes. Lane cursors as in the dense form above.
                auto stream = [&](auto wkc) {
                    constexpr int WK = decltype(wkc)::value;
                    int rcur = 0, pos = gl, pend = 0, jn = 0;
                    CandT cn;
                    bool vn = pos < total;
                    if (vn) {
                        while (rE[rcur] <= pos) ++rcur;
                        pend = rE[rcur];
                        jn = rA[rcur] + pos - (rcur ? rE[rcur - 1] : 0);
                        cn.load(A, jn);
                    }
                    for (int p0 = 0; p0 < total; p0 += G) {
                        const bool v = vn;
                        const int j = jn;
                        const CandT c = cn;
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
                        T dx[3] = {T(0), T(0), T(0)};
                        if (v) {
                            if constexpr (MIXED) {
                                float ddx, ddy, ddz = 0.f;
                                if (DIM == 2) {
                                    ddx = (c.h0.x - thi[0]) + (c.h0.z - tlo[0]);
                                    ddy = (c.h0.y - thi[1]) + (c.h0.w - tlo[1]);
                                } else {
                                    ddx = (c.h0.x - thi[0]) + (c.h0.w - tlo[0]);
                                    ddy = (c.h0.y - thi[1]) + (c.h1.x - tlo[1]);
                                    ddz = (c.h0.z - thi[2]) + (c.h1.y - tlo[2]);
                                }
                                float d2f = ddx * ddx + ddy * ddy;
                                if (DIM == 3) d2f += ddz * ddz;
                                int cl;
                                if constexpr (WK == PCMS_WENDLAND_C2)   // classify32 for this kind
                                    cl = d2f > r2f * (1.0f + MIX_BAND)
                                             ? 0
                                             : (d2f < r2f * (1.0f - MIX_BAND) ? 1 : -1);
                                else
                                    cl = classify32(A.weight, d2f, r2f);
                                if (cl < 0) {
                                    double te[3] = {0.0, 0.0, 0.0};
#pragma unroll
                                    for (int d = 0; d < DIM; d++) te[d] = A.tx64[d * A.nt + t];
                                    cl = select_exact(A.weight, dist2_exact<DIM>(A.sx64, A.ns, j, te),
                                                      r, r2);
                                }
                                in = cl != 0;
                                dx[0] = (T)ddx;
                                dx[1] = (T)ddy;
                                dx[2] = (T)ddz;
                            } else {
                                const double e0 = __dsub_rn(c.x[0], tx[0]);
                                const double e1 = __dsub_rn(c.x[1], tx[1]);
                                double d2 = __dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1));
                                double e2 = 0.0;
                                if (DIM == 3) {
                                    e2 = __dsub_rn(c.x[2], tx[2]);
                                    d2 = __dadd_rn(d2, __dmul_rn(e2, e2));
                                }
                                in = select64(A.weight, d2, r, r2, r2_in);
                                dx[0] = (T)e0;
                                dx[1] = (T)e1;
                                dx[2] = (T)e2;
                            }
                        }
                        const unsigned bal = __ballot_sync(gmask, in) & gmask;
                        const int nin = __popc(bal);
                        if (MODE == MODE_COUNT) {
                            cnt += nin;
                            continue;
                        }
                        if (in) {
                            T pay;
                            if constexpr (MODE == MODE_MAP) pay = pack_index(j, T(0));
                            else pay = (T)c.f;
                            const int qp = (head + qn + __popc(bal & lt)) & (QCAP - 1);
                            q[qp] = make_entry<T>(dx[0], dx[1], dx[2], pay);
                        }
                        qn += nin;
                        cnt += nin;
                        __syncwarp(gmask);
                        if (qn >= G) {
                            QE e = q[(head + gl) & (QCAP - 1)];
                            T edx[3] = {e.x, e.y, e.z};
                            accumulate<DIM, DEG, MODE, T, NACC, WK>(acc, edx, e.w, A.weight, inv_r, bc);
                            if constexpr (ACC == ACC_BK) {
                                if (++pops == BK_BLOCK) {
                                    tot.flush(acc);
                                    pops = 0;
                                }
                            }
                            if (MODE == MODE_MAP) {
                                if (one_pass) {
                                    if (written + gl < STG) stg[written + gl] = unpack_index(e.w);
                                } else if (A.cols && written + gl < row_len) {
                                    A.cols[row_off + written + gl] = unpack_index(e.w);
                                }
                                written += G;
                            }
                            head = (head + G) & (QCAP - 1);
                            qn -= G;
                            __syncwarp(gmask);
                        }
                    }
                };
                if (MIXED && MODE != MODE_COUNT && A.weight == PCMS_WENDLAND_C2)
                    stream(std::integral_constant<int, PCMS_WENDLAND_C2>{});
                else
                    stream(std::integral_constant<int, -1>{});
                __syncwarp(gmask);   // the row table is rewritten by the next RB rows
            }
            if constexpr (PRED) cnt = __reduce_add_sync(gmask, (unsigned)cnt);   // lanes' counts
            if (MODE != MODE_COUNT && qn > 0) {
                if (gl < qn) {
                    QE e = q[(head + gl) & (QCAP - 1)];
                    T edx[3] = {e.x, e.y, e.z};
                    accumulate<DIM, DEG, MODE, T, NACC>(acc, edx, e.w, A.weight, inv_r, bc);
                    if (MODE == MODE_MAP) {
                        if (one_pass) {
                            if (written + gl < STG) stg[written + gl] = unpack_index(e.w);
                        } else if (A.cols && written + gl < row_len) {
                            A.cols[row_off + written + gl] = unpack_index(e.w);
                        }
                    }
                }
                __syncwarp(gmask);
            }
            if (MODE != MODE_MAP && A.need > 0 && cnt < A.need && k < MAX_DOUBLINGS && cnt < A.ns) {
                ++k;
                continue;
            }
            break;
        }
        MT red[NA];
        if constexpr (SMEM_TOT) {
            // The totals are in shared memory: lane i reduces running sum i over the warp's 32
            // lanes (TwoSum on the leading parts, plain sums of the trailing parts), starting
            // at lane i so that the lanes' reads fall in different banks, and stores it.
            tot.flush(acc);
            __syncwarp();
            if (NACC > 0 && gl < NACCP) {
                MT* dst = (MT*)A.mom + (A.list ? wk : t) * NACCP;   // list mode: by list position
                if (gl < NACC) {
                    const float2* col = &tot_s[gl * 256 + (threadIdx.x & ~31)];
                    float hi = 0.f, lo = 0.f;
                    for (int m = 0; m < 32; m++) {
                        const float2 v = col[(m + gl) & 31];   // a lane's total is v.x - v.y
                        float sm, e;
                        two_sum32(hi, v.x, sm, e);
                        lo = (lo - v.y) + e;
                        hi = sm;
                    }
                    dst[gl] = make_float2(hi, lo);
                } else {
                    dst[gl] = MT{};
                }
            }
            __syncwarp();   // the next target clears the totals
        } else if constexpr (ACC == ACC_BK) {
            // the lane's total is sum - cmp; reduce the pairs (hi, lo) = (sum, -cmp) with
            // TwoSum on the leading parts and plain sums of the trailing parts
            tot.flush(acc);
#pragma unroll
            for (int i = 0; i < NA; i++) {
                const float2 hl = tot.pair(i);
                float hi = hl.x, lo = hl.y;
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    const float ho = __shfl_xor_sync(gmask, hi, o);
                    const float lw = __shfl_xor_sync(gmask, lo, o);
                    float s, e;
                    two_sum32(hi, ho, s, e);
                    lo = (lo + lw) + e;
                    hi = s;
                }
                red[i] = make_float2(hi, lo);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NA; i++) {
                red[i] = acc[i];
                if (NACC > 0) {
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) red[i] += __shfl_xor_sync(gmask, red[i], o);
                }
            }
        }
        if (gl == 0) {
            if (NACC > 0 && !SMEM_TOT) {
                MT* dst = (MT*)A.mom + (A.list ? wk : t) * NACCP;   // list mode: by list position
#pragma unroll
                for (int i = 0; i < NACCP; i++) {
                    if (i < NACC) dst[i] = red[i < NACC ? i : 0];
                    else dst[i] = MT{};
                }
            }
            A.counts[t] = cnt;
            if (A.kexp_out) A.kexp_out[t] = k;
            if constexpr (MIXED && ACC == ACC_BK && MODE != MODE_COUNT) {
                if (A.basis_out && !A.list)
                    A.basis_out[t] = make_float4(bcv[0], bcv[1], bcv[2], bcv[3]);
            }
            if (MODE == MODE_MAP && !one_pass && A.cols && cnt != row_len) atomicOr(A.err, 1u);
        }
        if (MODE == MODE_MAP && one_pass) {
            // reserve the row, then copy the staged columns (or leave the row to the second walk)
            unsigned long long base = 0;
            if (gl == 0) base = atomicAdd(A.nnz_ctr, (unsigned long long)cnt);
            base = __shfl_sync(gmask, base, 0, G);
            const bool fits = cnt <= STG && (int64_t)(base + cnt) <= A.cols_cap;
            __syncwarp(gmask);
            if (fits)
                for (int i = gl; i < cnt; i += G) A.cols[base + i] = stg[i];
            if (gl == 0) {
                A.offsets[t] = (int64_t)base;
                if (!fits) A.redo[atomicAdd(A.n_redo, 1)] = (int32_t)t;
            }
            __syncwarp(gmask);   // the stage is reused by the group's next target
        }
    }
}

// ------------------------------------------------------------------------------------
// per-target solve: G from the moments (+ lambda on the diagonal), LDL^T with the pivot
// guard d_k > tau * G_kk for every k (d_k / G_kk = R_kk^2 / ||column k||^2 of the weighted
// Vandermonde matrix), then
//   y[0..m) = G^-1 a_t   (L w = a_t, z = D^-1 w, L^T y = z; the operator row is w a^T y)
//   *c0     = y^T g = a_t^T G^-1 g   (MODE_FUSED; G is symmetric)
// with a_t = a(u_t) the basis at the target: e_1 in the target-centred basis (at = null),
// or a(-c/s) in a re-centred one.
//   *amp    = sqrt(G_00) sum_k |y_k| sqrt(G_kk): how much relative perturbations of the
//             moments are amplified in c_0 (1 for an orthogonal basis).
// mom = [moments of degree <= 2k (graded-lex)] [g (FUSED only)]. Returns false when the
// guard fails. Host-callable so the algebra can be checked without a GPU.
// ------------------------------------------------------------------------------------
// *rho (optional) = min_k d_k / G_kk, the smallest pivot ratio: about 1 / cond of the
// diagonally scaled G. An error e in the moments moves c_0 by up to about e amp / rho.
template <int DIM, int DEG, int MODE>
__host__ __device__ __forceinline__ bool solve_moments(const double* mom, double lambda,
                                                       double tau, double* out, double* c0,
                                                       double* amp, const double* at = nullptr,
                                                       double* rho = nullptr) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NP = M * (M + 1) / 2;
    double L[NP];
    sfor<M>([&](auto K) {
        constexpr int k = decltype(K)::value;
        sfor<k + 1>([&](auto Lx) {
            constexpr int l = decltype(Lx)::value;
            constexpr int kl = mono_prod(DIM, k, l);   // evaluated at compile time
            L[k * (k + 1) / 2 + l] = mom[kl] + (k == l ? lambda : 0.0);
        });
    });
    double invd[M], diag[M];
    bool ok = true;
    sfor<M>([&](auto K) {
        constexpr int k = decltype(K)::value;
        diag[k] = L[k * (k + 1) / 2 + k];
        sfor<k>([&](auto Jx) {
            constexpr int j = decltype(Jx)::value;
            double s = L[k * (k + 1) / 2 + j];
            sfor<j>([&](auto Ix) {
                constexpr int i = decltype(Ix)::value;
                s -= L[k * (k + 1) / 2 + i] * (L[j * (j + 1) / 2 + i] * L[i * (i + 1) / 2 + i]);
            });
            L[k * (k + 1) / 2 + j] = s * invd[j];
        });
        const double gkk = L[k * (k + 1) / 2 + k];
        double dk = gkk;
        sfor<k>([&](auto Jx) {
            constexpr int j = decltype(Jx)::value;
            const double lkj = L[k * (k + 1) / 2 + j];
            dk -= lkj * lkj * L[j * (j + 1) / 2 + j];
        });
        ok = ok && (dk > tau * gkk);
        if (rho) *rho = k == 0 ? dk / gkk : fmin(*rho, dk / gkk);
        L[k * (k + 1) / 2 + k] = dk;
        invd[k] = recip64(dk);
    });
    if (!ok) return false;
    {
        double w[M], z[M];
        sfor<M>([&](auto K) {
            constexpr int k = decltype(K)::value;
            double a = at ? at[k] : (k == 0 ? 1.0 : 0.0);
            sfor<k>([&](auto Jx) {
                constexpr int j = decltype(Jx)::value;
                a -= L[k * (k + 1) / 2 + j] * w[j];
            });
            w[k] = a;
            z[k] = a * invd[k];
        });
        sfor<M>([&](auto K) {
            constexpr int k = M - 1 - decltype(K)::value;
            double a = z[k];
            sfor<M - 1 - k>([&](auto Jx) {
                constexpr int j = k + 1 + decltype(Jx)::value;
                a -= L[j * (j + 1) / 2 + k] * out[j];
            });
            out[k] = a;
        });
    }
    double cc = 0.0;
    for (int k = 0; k < M; k++)
        if (MODE == MODE_FUSED) cc += out[k] * mom[NM + k];
    if (c0) *c0 = cc;
    if (amp) {   // an error estimate for routing: FP32 on the device (overflow gives inf: routed on)
#ifdef __CUDA_ARCH__
        float sf = 0.f;
        for (int k = 0; k < M; k++) sf += fabsf((float)out[k]) * sqrtf(fmaxf((float)diag[k], 0.f));
        *amp = (double)(sf * sqrtf(fmaxf((float)diag[0], 0.f)));
#else
        double sd = 0.0;
        for (int k = 0; k < M; k++) sd += fabs(out[k]) * sqrt(fmax(diag[k], 0.0));
        *amp = sd * sqrt(fmax(diag[0], 0.0));
#endif
    }
    return true;
}

// ------------------------------------------------------------------------------------
// k_solve: one thread per target
// ------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ double mom_value(float v) { return (double)v; }
__host__ __device__ __forceinline__ double mom_value(double v) { return v; }
__host__ __device__ __forceinline__ double mom_value(float2 v) { return (double)v.x + (double)v.y; }

__host__ __device__ __forceinline__ bool is_target_centred(float4 b) {
    return b.x == 0.f && b.y == 0.f && b.z == 0.f && b.w == 1.f;
}

// Re-centred basis from target-centred moments (offsets in units of r): c = weighted
// centroid, s = weighted root-mean-square distance from c per coordinate; returned as
// (c, 1/s) rounded to FP32. Falls back to the target-centred basis when the spread is zero.
template <int DIM>
__host__ __device__ inline float4 recentre_basis(const double* mom) {
    const double w0 = mom[0];
    double c[3] = {0.0, 0.0, 0.0};
    double var = 0.0;
    sfor<DIM>([&](auto D) {
        constexpr int d = decltype(D)::value;
        constexpr int i1 = mono_index(DIM, d == 0, d == 1, d == 2);
        constexpr int i2 = mono_index(DIM, 2 * (d == 0), 2 * (d == 1), 2 * (d == 2));
        c[d] = mom[i1] / w0;
        var += mom[i2] / w0 - c[d] * c[d];
    });
    const double s2 = var / DIM;
    if (!(w0 > 0.0) || !(s2 > 1e-12)) return make_float4(0.f, 0.f, 0.f, 1.f);
    return make_float4((float)c[0], (float)c[1], (float)c[2], (float)(1.0 / sqrt(s2)));
}

// The re-centred basis for moments that were assembled in the basis b = (c_b, 1/s_b): their
// weighted centroid c' and spread s' (offsets in b) give c = c_b + s_b c' and
// 1/s = (1/s_b) (1/s'), rounded to FP32. From the identity this is recentre_basis itself.
template <int DIM>
__host__ __device__ inline float4 recentre_from(float4 b, const double* mom) {
    const float4 r = recentre_basis<DIM>(mom);
    if (is_target_centred(b)) return r;
    if (is_target_centred(r)) return b;   // no usable spread in b: keep b
    const double sb = 1.0 / (double)b.w;
    return make_float4((float)((double)b.x + sb * (double)r.x),
                       (float)((double)b.y + sb * (double)r.y),
                       (float)((double)b.z + sb * (double)r.z), (float)((double)b.w * (double)r.w));
}

// a(u'_t), the basis at the target in the basis b: u'_t = (0 - c) / s with the FP32 (c, 1/s)
template <int DIM, int DEG>
__host__ __device__ inline void basis_at_target(float4 b, double* at) {
    constexpr int M = mono_count(DIM, DEG);
    const double ut[3] = {-(double)b.x * (double)b.w, -(double)b.y * (double)b.w,
                          -(double)b.z * (double)b.w};
    at[0] = 1.0;
    sfor<M - 1>([&](auto I) {
        constexpr int p = decltype(I)::value + 1;
        at[p] = at[mono_parent(DIM, p)] * ut[mono_var(DIM, p)];
    });
}

// The mixed tiers' solve without FP64 arithmetic. G y = a_t is solved by iterative refinement:
// an FP32 LDL^T of G's leading FP32 parts gives each correction, and every residual
// a_t - G y is formed in double-FP32 arithmetic (TwoProduct by FMA, TwoSum) from the moments
// as stored (plain FP32 sums are exact FP32 values; blocked sums are FP32 pairs), with y kept
// as an FP32 pair. An error e in y moves c_0 (and an operator row's value) by about e amp, so
// the refinement runs until a correction is below 2^-20 / amp of y: c_0 then moves by at most
// 2^-20 of the field, 5% of the 2e-5 bound, next to the moments' own FP32 error that the
// tiers' amp bounds keep below a third of it. The attainable accuracy is about
// kappa amp 2^-48 (the residual's double-FP32 error relative to |G| |y|).
// Returns
//   1  solved: y = yh + yl, *c0 (FUSED) and *amp as solve_moments;
//   2  not refined, because amp (from the FP32 solve) exceeds amp_accept, the tier's
//      acceptance bound, by more than the FP32 solve's error: the caller hands the target on;
//   0  declined: a pivot of the FP32 factorization is not above 1e-4 G_kk, which exceeds every
//      guard's threshold by more than the FP32 factorization's error (about 2 m 2^-24 G_kk),
//      or REFINE_STEPS steps do not converge. The caller then solves in FP64, so a target
//      accepted here is one the FP64 guard accepts, and decisions near a threshold are the
//      FP64 factorization's.
__host__ __device__ __forceinline__ float mom_hi(float v) { return v; }
__host__ __device__ __forceinline__ float mom_lo(float) { return 0.f; }
__host__ __device__ __forceinline__ float mom_hi(float2 v) { return v.x; }
__host__ __device__ __forceinline__ float mom_lo(float2 v) { return v.y; }
__host__ __device__ __forceinline__ float rcp32(float x) {
#ifdef __CUDA_ARCH__
    return __frcp_rn(x);
#else
    return 1.f / x;
#endif
}

constexpr int REFINE_STEPS = 6;
constexpr float REFINE_PIVOT = 1e-4f;

template <int DIM, int DEG, int MODE, typename MT>
__host__ __device__ __forceinline__ int solve_moments_refined(const MT* mt, const double* at,
                                                              float amp_accept, float* yh,
                                                              float* yl, double* c0,
                                                              float* amp) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NP = M * (M + 1) / 2;
    float L[NP];
    sfor<M>([&](auto K) {
        constexpr int k = decltype(K)::value;
        sfor<k + 1>([&](auto Lx) {
            constexpr int l = decltype(Lx)::value;
            constexpr int kl = mono_prod(DIM, k, l);
            L[k * (k + 1) / 2 + l] = mom_hi(mt[kl]);
        });
    });
    float invd[M], diag[M];
    bool ok = true;
    sfor<M>([&](auto K) {
        constexpr int k = decltype(K)::value;
        diag[k] = L[k * (k + 1) / 2 + k];
        sfor<k>([&](auto Jx) {
            constexpr int j = decltype(Jx)::value;
            float sv = L[k * (k + 1) / 2 + j];
            sfor<j>([&](auto Ix) {
                constexpr int i = decltype(Ix)::value;
                sv -= L[k * (k + 1) / 2 + i] * (L[j * (j + 1) / 2 + i] * L[i * (i + 1) / 2 + i]);
            });
            L[k * (k + 1) / 2 + j] = sv * invd[j];
        });
        float dk = L[k * (k + 1) / 2 + k];
        sfor<k>([&](auto Jx) {
            constexpr int j = decltype(Jx)::value;
            const float lkj = L[k * (k + 1) / 2 + j];
            dk -= lkj * lkj * L[j * (j + 1) / 2 + j];
        });
        ok = ok && (dk > REFINE_PIVOT * diag[k]);
        L[k * (k + 1) / 2 + k] = dk;
        invd[k] = rcp32(dk);
    });
    if (!ok) return 0;
    // x = (L D L^T)^-1 b in FP32
    auto ldl_solve = [&](const float* b, float* x) {
        float w[M];
        sfor<M>([&](auto K) {
            constexpr int k = decltype(K)::value;
            float a = b[k];
            sfor<k>([&](auto Jx) {
                constexpr int j = decltype(Jx)::value;
                a -= L[k * (k + 1) / 2 + j] * w[j];
            });
            w[k] = a;
        });
        sfor<M>([&](auto K) {
            constexpr int k = M - 1 - decltype(K)::value;
            float a = w[k] * invd[k];
            sfor<M - 1 - k>([&](auto Jx) {
                constexpr int j = k + 1 + decltype(Jx)::value;
                a -= L[j * (j + 1) / 2 + k] * x[j];
            });
            x[k] = a;
        });
    };
    float ah[M], al[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        if (at) {
            ah[k] = (float)at[k];
            al[k] = (float)(at[k] - (double)ah[k]);
        } else {
            ah[k] = k == 0 ? 1.f : 0.f;
            al[k] = 0.f;
        }
    }
    ldl_solve(ah, yh);
    auto amp_of = [&]() {
        float sf = 0.f;
#pragma unroll
        for (int k = 0; k < M; k++) sf += fabsf(yh[k]) * sqrtf(fmaxf(diag[k], 0.f));
        return sf * sqrtf(fmaxf(diag[0], 0.f));
    };
    const float amp0 = amp_of();
    if (!(amp0 <= 1e30f)) return 0;
    if (amp0 > 1.01f * amp_accept) {
        *amp = amp0;
        return 2;
    }
    const float tol = 9.5367431640625e-07f / fmaxf(amp0, 1.f);   // 2^-20 / amp
#pragma unroll
    for (int k = 0; k < M; k++) yl[k] = 0.f;
    bool conv = false;
    for (int it = 0; it < REFINE_STEPS && !conv; it++) {
        float rh[M];
        sfor<M>([&](auto K) {
            constexpr int k = decltype(K)::value;
            float sh = ah[k], sl = al[k];
            sfor<M>([&](auto Lx) {
                constexpr int l = decltype(Lx)::value;
                constexpr int kl = mono_prod(DIM, k, l);
                const MT g = mt[kl];
                const float gh = mom_hi(g), gll = mom_lo(g);
                const float ph = gh * yh[l];
                const float pl = fmaf(gh, yh[l], -ph) + (gh * yl[l] + gll * yh[l]);
                float s2, e2;
                two_sum32(sh, -ph, s2, e2);
                sl = (sl - pl) + e2;
                sh = s2;
            });
            rh[k] = sh + sl;
        });
        float dy[M];
        ldl_solve(rh, dy);
        float dmax = 0.f, ymax = 0.f;
#pragma unroll
        for (int k = 0; k < M; k++) {
            float s2, e2;
            two_sum32(yh[k], dy[k], s2, e2);
            const float lo = yl[k] + e2;
            yh[k] = s2 + lo;
            yl[k] = lo - (yh[k] - s2);
            dmax = fmaxf(dmax, fabsf(dy[k]));
            ymax = fmaxf(ymax, fabsf(yh[k]));
        }
        conv = dmax <= tol * ymax;
    }
    if (!conv) return 0;
    if (MODE == MODE_FUSED) {   // c_0 = y^T g, g the right-hand side moments, as a pair
        float ch = 0.f, cl = 0.f;
#pragma unroll
        for (int k = 0; k < M; k++) {
            const MT g = mt[NM + k];
            const float gh = mom_hi(g), gll = mom_lo(g);
            const float ph = gh * yh[k];
            const float pl = fmaf(gh, yh[k], -ph) + (gh * yl[k] + gll * yh[k]);
            float s2, e2;
            two_sum32(ch, ph, s2, e2);
            cl = (cl + pl) + e2;
            ch = s2;
        }
        *c0 = (double)ch + (double)cl;
    }
    *amp = amp_of();
    return 1;
}

// A tier's acceptance bound on amp for a target of n neighbours (the tier table above),
// evaluated in FP32: the bound is a calibrated constant, not a precision-critical quantity.
// dense: tier 1 of a dense one-shot plan (blocks of BK_BLOCK_DENSE pairs).
__host__ __device__ __forceinline__ float amp_bound(int acc, int n, int group, bool dense = false) {
    const float nf = (float)n;
    if (acc == ACC_PLAIN) {
        const float g = (float)group;
        return (float)AMP_T1 / (1.f + sqrtf(nf / (3.f * g * g)));
    }
    return (float)(dense ? AMP_BK_DENSE : AMP_BK) * sqrtf(nf);
}

// PASS: 0 = FP64 moments (one FP64 solve); for FP32 moments (the mixed tiers) 1 = the refined
// FP32 solve, whose declined work items go to fb_list, and 2 = the FP64 solve of those items.
// Two launches keep the FP64 solve's registers out of the refined pass.
template <int DIM, int DEG, int MODE, typename MT, int PASS = 0>
__global__ void __launch_bounds__(128, PASS == 1 ? 3 : 1) k_solve(SolveArgs S) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NACC = MODE == MODE_FUSED ? NM + M : NM;
    constexpr int NACCP = round_up4(NACC);
    static_assert((PASS == 0) == std::is_same<MT, double>::value, "passes: FP32 moments only");
    const int64_t nwork = PASS == 2 ? (int64_t)(*S.n_fb) : (S.list ? (int64_t)(*S.n_list) : S.nt);
    // tier 1 of a dense one-shot plan was assembled in blocks of BK_BLOCK_DENSE pairs
    const bool dense =
        DIM == 2 && MODE == MODE_FUSED && S.tier == 1 && S.acc == ACC_BK && S.group == 32;
    for (int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ii < nwork;
         ii += (int64_t)gridDim.x * blockDim.x) {
        const int64_t wk = PASS == 2 ? (int64_t)S.fb_list[ii] : ii;
        const int64_t t = S.list ? (int64_t)S.list[wk] : wk;
        const int cnt = S.counts[t];
        int st = PCMS_TARGET_OK;
        double val = 0.0, amp = 0.0, rho = 1.0;
        float amp32 = 0.f;   // amp for routing and row flags (the refined pass works in FP32)
        double y[M];
        double mom[NACC];
        float yh[M], yl[M];   // the refined FP32 solve's y (mixed tiers), as pairs
        bool refined = false;
        float4 bas = make_float4(0.f, 0.f, 0.f, 1.f);
        bool recentred = false;
        const MT* src = (const MT*)S.mom + (S.list ? wk : t) * NACCP;
        if (cnt < M) {
            st = PCMS_TARGET_UNDERDETERMINED;
        } else {
            double at[M];
            if (S.basis_in) {
                bas = S.basis_in[wk];
                recentred = !is_target_centred(bas);
                if (recentred) basis_at_target<DIM, DEG>(bas, at);
                if (PASS != 2 && recentred && S.n_recentred) atomicAdd(S.n_recentred, 1);
            }
            if constexpr (PASS == 1) {
                int rs = 0;
                if (S.lambda == 0.0) {
                    rs = solve_moments_refined<DIM, DEG, MODE, MT>(
                        src, recentred ? at : nullptr, amp_bound(S.acc, cnt, S.group, dense), yh, yl,
                        &val, &amp32);
                }
                if (rs == 0) {   // the FP64 pass solves it
                    S.fb_list[atomicAdd(S.n_fb, 1)] = (int32_t)wk;
                    continue;
                }
                refined = true;
            } else {
#pragma unroll
                for (int i = 0; i < NACC; i++) mom[i] = mom_value(src[i]);
                if (!solve_moments<DIM, DEG, MODE>(mom, S.lambda, S.tau, y, &val, &amp,
                                                   recentred ? at : nullptr, &rho))
                    st = PCMS_TARGET_ILL_CONDITIONED;
                amp32 = (float)amp;
            }
        }
        if (S.tier == 4 && st != PCMS_TARGET_OK) {   // keep the first FP64 solve
            if (S.qr_list) S.qr_list[atomicAdd(S.n_qr, 1)] = (int32_t)t;
            continue;
        }
        const bool to_refine =
            S.tier == 3 && S.refine64 && st == PCMS_TARGET_OK && amp32 > (float)AMP_FP64;
        if (to_refine) {
            const int pos = atomicAdd(S.n2, 1);
            S.list2[pos] = (int32_t)t;
            S.basis2[pos] = recentre_basis<DIM>(mom);
        }
        if (S.qr_list && S.tier >= 3 && !to_refine && st == PCMS_TARGET_OK &&
            amp > (double)S.amp_qr * rho)
            S.qr_list[atomicAdd(S.n_qr, 1)] = (int32_t)t;
        if (S.tier < 3 && st != PCMS_TARGET_UNDERDETERMINED) {
            bool ok = st == PCMS_TARGET_OK;
            if (ok) ok = amp32 <= amp_bound(S.acc, cnt, S.group, dense);
            if (!ok) {
                // tier 2 only helps if it differs from this pass: a plain tier 1, or a
                // re-centred basis
                const bool to2 = S.tier == 1 && (S.acc == ACC_PLAIN || S.recentre);
                if (to2) {
                    const int pos = atomicAdd(S.n2, 1);
                    S.list2[pos] = (int32_t)t;
                    if (refined) {
#pragma unroll
                        for (int i = 0; i < NACC; i++) mom[i] = mom_value(src[i]);
                    }
                    if (S.basis2)
                        S.basis2[pos] = S.recentre ? recentre_from<DIM>(bas, mom)
                                                   : make_float4(0.f, 0.f, 0.f, 1.f);
                } else {
                    S.list3[atomicAdd(S.n3, 1)] = (int32_t)t;
                }
                continue;   // a later tier writes this target
            }
        }
        // operator rows: 0 = FP32; 1 = FP32 u, w as in the moments, exact FP32 monomial
        // products and a double-FP32 dot product with y;
        // 2 = everything in FP64 (tier 3: y belongs to the exact FP64 moments);
        // 3 = as 1 in the re-centred basis rc[t]; 4 = as 0 in the re-centred basis rc[t]
        if (MODE == MODE_MAP && S.flags) {
            const int flag = recentred ? (amp32 > (float)AMP_SHAPE ? 3 : 4)
                                       : (S.tier == 3 ? 2 : (amp32 > (float)AMP_SHAPE ? 1 : 0));
            S.flags[t] = (int8_t)flag;
            if (recentred && S.rc) S.rc[t] = bas;
            if (flag == 2 && S.list64) S.list64[atomicAdd(S.n64, 1)] = (int32_t)t;
        }
        const double nanv = __longlong_as_double(0x7ff8000000000000LL);
        if (MODE == MODE_FUSED) {
            const int64_t o = S.perm_t ? (int64_t)S.perm_t[t] : t;
            const double v = st == PCMS_TARGET_OK ? val : nanv;
            if (S.out_is_double) ((double*)S.out)[o] = v;
            else ((float*)S.out)[o] = (float)v;
            if (S.status) S.status[o] = (int8_t)st;
        } else if (refined) {
            // mixed rows of flags 0, 1, 3 and 4 read y as pairs only (k_shape)
#pragma unroll
            for (int k = 0; k < M; k++) S.yf[t * M + k] = make_float2(yh[k], yl[k]);
            S.status[t] = (int8_t)st;
        } else {
#pragma unroll
            for (int k = 0; k < M; k++) {
                const double yk = st == PCMS_TARGET_OK ? y[k] : nanv;
                S.y[t * M + k] = yk;
                if (S.yf) {
                    const float hi = (float)yk;
                    S.yf[t * M + k] = make_float2(hi, (float)(yk - (double)hi));
                }
            }
            S.status[t] = (int8_t)st;
        }
    }
}

// ------------------------------------------------------------------------------------
// k_shape: N_j = w_j a(u_j)^T y
// ------------------------------------------------------------------------------------
// Three blocks per SM (80 registers) for the stored mixed rows (3D quadratic: 20 bytes of
// spills, 3.9 -> 3.3 ms on the 8M operator) and for rows applied as evaluated of degree <= 1
// (2D linear, 16 fields: 0.217 -> 0.164 ms per 1M targets); quadratic rows applied as
// evaluated keep two (at 80 registers their spills cost more than the warps gain).
template <int DIM, int DEG, bool MIXED, int G, bool APPLY = false>
__global__ void __launch_bounds__(256, (APPLY && DEG <= 1) || (!APPLY && MIXED) ? 3 : 1) k_shape(ShapeArgs S) {
    static_assert(DEG <= 2, "operator rows: exact double-FP32 monomials need degree <= 2");
    static_assert(!APPLY || MIXED, "fused rows and apply: mixed maps");
    using T = typename std::conditional<MIXED, float, double>::type;
    constexpr int M = mono_count(DIM, DEG);
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gi = lane / G, gl = lane % G;
    const int64_t ngroups = (int64_t)gridDim.x * (blockDim.x >> 5) * GPW;
    const int64_t gid = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GPW + gi;
    const Grid& g = S.g;
    for (int64_t t = gid; t < S.nt; t += ngroups) {
        // the FP64 target coordinates serve the FP64 rows only; the FP32 pairs of y come from
        // the solve (one conversion per target instead of one per lane)
        double tx[3] = {0, 0, 0};
        float thi[3] = {0.f, 0.f, 0.f}, tlo[3] = {0.f, 0.f, 0.f};
        if constexpr (MIXED) load_hilo<DIM>(S.thl0, S.thl1, t, thi, tlo);
        // y as T, and for mixed maps also as an unevaluated FP32 pair (y = yh + yl to ~2^-48)
        T y[M];
        float yl[M];   // rows applied as evaluated read the trailing parts where they need them
#pragma unroll
        for (int k = 0; k < M; k++) {
            if constexpr (MIXED) {
                const float2 v = S.yf[t * M + k];
                y[k] = v.x;
                yl[k] = APPLY ? 0.f : v.y;
            } else {
                y[k] = S.y[t * M + k];
                yl[k] = 0.f;
            }
        }
        const int flag = S.flags ? S.flags[t] : 0;
        // FP64 target coordinates: FP64 paths, and the FP64-assembled rows (flag 2) of mixed
        // maps, which rows applied as evaluated leave to k_rows64_apply
        if (!MIXED || (!APPLY && flag == 2)) {
#pragma unroll
            for (int d = 0; d < DIM; d++) tx[d] = S.tx64[d * S.nt + t];
        }
        T bcv[4] = {T(0), T(0), T(0), T(1)};
        if (flag >= 3) {   // re-centred basis (mixed tiers 1 and 2, FP64 refine pass)
            const float4 b4 = S.rc[t];
            bcv[0] = b4.x;
            bcv[1] = b4.y;
            bcv[2] = b4.z;
            bcv[3] = b4.w;
        }
        const int kx = S.kexp[t];
        const double r = S.lv.r[kx];
        T inv_r;
        if constexpr (MIXED) inv_r = S.lv.inv_rf[kx];
        else inv_r = S.lv.inv_r[kx];
        const int64_t a = S.offsets[t], b = (APPLY && flag == 2) ? a : a + S.counts[t];
        // APPLY: this lane's share of the row applied to the fields. Rows of FP64-assembled
        // targets (flag 2) are left to k_rows64_apply, which accumulates them in FP64: their
        // operator values can be large with cancelling signs (extrapolating targets with
        // about m neighbours: sum_j |N_j| up to amp), where FP32 sums would lose the bound.
        float facc[16];
#pragma unroll
        for (int q = 0; q < 16; q++) facc[q] = 0.f;
        const int nvf = APPLY ? S.fp / 4 : 0;
        // APPLY: the pair's field row, loaded when the pair is taken up so that the gather
        // overlaps the evaluation of its value
        float4 fx[4];
        float f1 = 0.f;
        auto gather = [&](int j) {
            if constexpr (APPLY) {
                if (S.fp == 1) {
                    f1 = S.fs[j];
                } else {
                    const float4* row = reinterpret_cast<const float4*>(S.fs + (int64_t)j * S.fp);
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (q < nvf) fx[q] = row[q];
                }
            }
        };
        auto emit = [&](int64_t i, int j, T v) {
            if constexpr (APPLY) {
                if (S.fp == 1) {
                    facc[0] += (float)v * f1;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        if (q < nvf) {
                            facc[4 * q] += (float)v * fx[q].x;
                            facc[4 * q + 1] += (float)v * fx[q].y;
                            facc[4 * q + 2] += (float)v * fx[q].z;
                            facc[4 * q + 3] += (float)v * fx[q].w;
                        }
                    }
                }
            } else {
                ((T*)S.vals)[i] = v;
            }
        };
        // Software pipeline over the row (mixed path): the column two pairs ahead and the
        // coordinates of the next pair are loaded before the current pair is evaluated, so
        // the gathers overlap the arithmetic instead of stalling on it.
        int64_t i = a + gl;
        int jc = i < b ? S.cols[i] : 0;
        int jn = i + G < b ? S.cols[i + G] : 0;
        float4 hc0 = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 hc1 = make_float2(0.f, 0.f);
        if (MIXED && i < b) {
            hc0 = S.hl0[jc];
            if (DIM == 3) hc1 = S.hl1[jc];
        }
        for (; i < b; i += G) {
            const int j = jc;
            gather(j);
            const float4 cur0 = hc0;
            const float2 cur1 = hc1;
            if (MIXED && i + G < b) {
                hc0 = S.hl0[jn];
                if (DIM == 3) hc1 = S.hl1[jn];
            }
            jc = jn;
            jn = i + 2 * G < b ? S.cols[i + 2 * G] : 0;
            if (MIXED && flag == 2) {
                // row of an FP64-assembled target: the exact FP64 offsets, weight and basis
                double e[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int d = 0; d < DIM; d++) e[d] = S.sx64[d * S.ns + j] - tx[d];
                double d2 = e[0] * e[0] + e[1] * e[1];
                if (DIM == 3) d2 += e[2] * e[2];
                const double ir = S.lv.inv_r[kx];
                const double w64 = weight_value<double>(S.weight, sqrt(d2) * ir);
                const double uu[3] = {e[0] * ir, e[1] * ir, e[2] * ir};
                double am[M];
                am[0] = 1.0;
                double s = S.y[t * M];
                sfor<M - 1>([&](auto I) {
                    constexpr int p = decltype(I)::value + 1;
                    constexpr int par = mono_parent(DIM, p);
                    constexpr int v = mono_var(DIM, p);
                    am[p] = am[par] * uu[v];
                    s += am[p] * S.y[t * M + p];
                });
                emit(i, j, (T)(w64 * s));
                continue;
            }
            T dx[3] = {T(0), T(0), T(0)};
            if (MIXED) {
                const float4 h0 = cur0;
                if (DIM == 2) {
                    dx[0] = (h0.x - thi[0]) + (h0.z - tlo[0]);
                    dx[1] = (h0.y - thi[1]) + (h0.w - tlo[1]);
                } else {
                    const float2 h1 = cur1;
                    dx[0] = (h0.x - thi[0]) + (h0.w - tlo[0]);
                    dx[1] = (h0.y - thi[1]) + (h1.x - tlo[1]);
                    dx[2] = (h0.z - thi[2]) + (h1.y - tlo[2]);
                }
            } else {
#pragma unroll
                for (int d = 0; d < DIM; d++) dx[d] = (T)(S.sx64[d * S.ns + j] - tx[d]);
            }
            T d2 = dx[0] * dx[0] + dx[1] * dx[1];
            if (DIM == 3) d2 += dx[2] * dx[2];
            T qv;
            if constexpr (MIXED) qv = sqrt_approx(d2) * inv_r;
            else qv = sqrt(d2) * inv_r;
            const T w = weight_value<T>(S.weight, qv);
            T u[3];
            basis_offsets<DIM, T>(dx, inv_r, flag >= 3 ? bcv : nullptr, u);
            if constexpr (MIXED) {
                if (flag == 1 || flag == 3) {
                    // sensitive row (1), or a row in a re-centred basis (3): the same FP32 u
                    // and w as the moments; the monomials (degree <= 2) as exact FP32 pairs
                    // (TwoProduct by FMA) and the dot product with y in double-FP32
                    // arithmetic (TwoProduct terms, TwoSum accumulation, ~2^-48), since y's
                    // entries cancel when amp is large
                    float ah[M], al[M];
                    ah[0] = 1.f;
                    al[0] = 0.f;
                    sfor<M - 1>([&](auto I) {
                        constexpr int p = decltype(I)::value + 1;
                        constexpr int par = mono_parent(DIM, p);
                        constexpr int v = mono_var(DIM, p);
                        if constexpr (par == 0) {
                            ah[p] = u[v];
                            al[p] = 0.f;
                        } else {   // degree 2: parent of degree 1 is an exact FP32 value
                            ah[p] = __fmul_rn(ah[par], u[v]);
                            al[p] = __fmaf_rn(ah[par], u[v], -ah[p]);
                        }
                    });
                    float sh = 0.f, sl = 0.f;
#pragma unroll
                    for (int k = 0; k < M; k++) {
                        const float ph = __fmul_rn(ah[k], y[k]);
                        const float ylk = APPLY ? S.yf[t * M + k].y : yl[k];
                        const float pl = __fmaf_rn(ah[k], y[k], -ph) + (ah[k] * ylk + al[k] * y[k]);
                        float s2, e2;
                        two_sum32(sh, ph, s2, e2);
                        sl = (sl + pl) + e2;
                        sh = s2;
                    }
                    emit(i, j, (T)(w * sh + w * sl));
                    continue;
                }
            }
            T am[M];
            am[0] = T(1);
            T s = y[0];
            sfor<M - 1>([&](auto I) {
                constexpr int p = decltype(I)::value + 1;
                constexpr int par = mono_parent(DIM, p);
                constexpr int v = mono_var(DIM, p);
                am[p] = am[par] * u[v];
                s += am[p] * y[p];
            });
            emit(i, j, w * s);
        }
        if constexpr (APPLY) {
            const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
            const int nacc = S.fp == 1 ? 1 : 4 * nvf;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                if (q < nacc) {
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) facc[q] += __shfl_xor_sync(gmask, facc[q], o);
                }
            }
            if (gl == 0) {
                const bool ok = S.status[t] == PCMS_TARGET_OK;
                const float nanf = __int_as_float(0x7fc00000);
                if (S.fp == 1) {
                    S.stage[t] = ok ? facc[0] : nanf;
                } else {
                    float4* dst = reinterpret_cast<float4*>(S.stage + t * S.fp);
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (q < nvf)
                            dst[q] = ok ? make_float4(facc[4 * q], facc[4 * q + 1], facc[4 * q + 2],
                                                      facc[4 * q + 3])
                                        : make_float4(nanf, nanf, nanf, nanf);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// k_rows64_apply: the fused apply of the FP64-assembled targets (flag 2, listed by the
// solve): each row evaluated in FP64 (exact offsets, weight, basis, the FP64 y) and applied
// to the fields with FP64 sums; the result replaces the target's staged row. A group of G
// lanes per listed target.
// ------------------------------------------------------------------------------------
template <int DIM, int DEG, int G>
__global__ void __launch_bounds__(256) k_rows64_apply(ShapeArgs S, const int32_t* __restrict__ list,
                                                      const int32_t* __restrict__ n_list) {
    constexpr int M = mono_count(DIM, DEG);
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gi = lane / G, gl = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
    const int64_t ngroups = (int64_t)gridDim.x * (blockDim.x >> 5) * GPW;
    const int64_t n = *n_list;
    for (int64_t e = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GPW + gi; e < n; e += ngroups) {
        const int64_t t = list[e];
        double tx[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < DIM; d++) tx[d] = S.tx64[d * S.nt + t];
        double y[M];
#pragma unroll
        for (int k = 0; k < M; k++) y[k] = S.y[t * M + k];
        const double ir = S.lv.inv_r[S.kexp[t]];
        const int64_t a = S.offsets[t], b = a + S.counts[t];
        double acc[16];
#pragma unroll
        for (int q = 0; q < 16; q++) acc[q] = 0.0;
        for (int64_t i = a + gl; i < b; i += G) {
            const int j = S.cols[i];
            double dx[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int d = 0; d < DIM; d++) dx[d] = S.sx64[d * S.ns + j] - tx[d];
            double d2 = dx[0] * dx[0] + dx[1] * dx[1];
            if (DIM == 3) d2 += dx[2] * dx[2];
            const double w = weight_value<double>(S.weight, sqrt(d2) * ir);
            const double u[3] = {dx[0] * ir, dx[1] * ir, dx[2] * ir};
            double am[M];
            am[0] = 1.0;
            double sum = y[0];
            sfor<M - 1>([&](auto I) {
                constexpr int p = decltype(I)::value + 1;
                am[p] = am[mono_parent(DIM, p)] * u[mono_var(DIM, p)];
                sum += am[p] * y[p];
            });
            const double v = w * sum;
            if (S.fp == 1) {
                acc[0] += v * (double)S.fs[j];
            } else {
                const float4* row = reinterpret_cast<const float4*>(S.fs + (int64_t)j * S.fp);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (4 * q < S.fp) {
                        const float4 x = row[q];
                        acc[4 * q] += v * (double)x.x;
                        acc[4 * q + 1] += v * (double)x.y;
                        acc[4 * q + 2] += v * (double)x.z;
                        acc[4 * q + 3] += v * (double)x.w;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 16; q++) {
            if (q < S.fp) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(gmask, acc[q], o);
            }
        }
        if (gl == 0 && S.status[t] == PCMS_TARGET_OK) {
#pragma unroll
            for (int q = 0; q < 16; q++)
                if (q < S.fp) S.stage[t * S.fp + q] = (float)acc[q];
        }
    }
}

}  // namespace pcms
