// Host-compiled harness for the CPU tests: exposes the library's per-target MLS algebra
// (the moment accumulation and the guarded LDL^T solve from mls_kernels.cuh, compiled for
// the host with T = double) so its arithmetic can be checked against numpy without a GPU.
// The FP32 form compiled here forms the moment terms one at a time; the device build forms
// the same products on two-lane FP32 instructions, with one fused multiply-add for each
// term of the top degree, which changes roundings but not the error model checked here.
#include "mls_kernels.cuh"

using namespace pcms;

template <int DIM, int DEG, int MODE>
static void accumulate_all(int kind, int n, const double* dx, const double* b, double inv_r,
                           const double* bc, double* acc) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NACC = MODE == MODE_FUSED ? NM + M : NM;
    double a[NACC];
    for (int i = 0; i < NACC; i++) a[i] = 0.0;
    for (int i = 0; i < n; i++)
        accumulate<DIM, DEG, MODE, double, NACC>(a, dx + 3 * i, b ? b[i] : 0.0, kind, inv_r, bc);
    for (int i = 0; i < NACC; i++) acc[i] = a[i];
}

// recentre = 1: a first target-centred pass gives the basis (recentre_basis), the moments
// are re-accumulated in it and the solve evaluates at a(u'_t); out then also holds the
// basis after y/c0 and amp (4 values) and, in map mode, the operator row N_j for each pair.
template <int DIM, int DEG, int MODE>
static int run(int kind, int n, const double* dx, const double* b, double inv_r, double lambda,
               double tau, double* mom_out, double* out, int recentre, double* rows) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NACC = MODE == MODE_FUSED ? NM + M : NM;
    double acc[NACC];
    accumulate_all<DIM, DEG, MODE>(kind, n, dx, b, inv_r, nullptr, acc);
    float4 bas = make_float4(0.f, 0.f, 0.f, 1.f);
    double at[M];
    const double* atp = nullptr;
    double bcv[4] = {0.0, 0.0, 0.0, 1.0};
    if (recentre) {
        bas = recentre_basis<DIM>(acc);
        bcv[0] = bas.x; bcv[1] = bas.y; bcv[2] = bas.z; bcv[3] = bas.w;
        accumulate_all<DIM, DEG, MODE>(kind, n, dx, b, inv_r, bcv, acc);
        basis_at_target<DIM, DEG>(bas, at);
        atp = at;
    }
    for (int i = 0; i < NACC; i++) mom_out[i] = acc[i];
    double y[M], c0 = 0.0, amp = 0.0;
    const bool ok = solve_moments<DIM, DEG, MODE>(acc, lambda, tau, y, &c0, &amp, atp);
    if (MODE == MODE_FUSED) out[0] = c0;
    else
        for (int k = 0; k < M; k++) out[k] = y[k];
    out[M] = amp;
    out[M + 1] = bas.x; out[M + 2] = bas.y; out[M + 3] = bas.z; out[M + 4] = bas.w;
    if (MODE == MODE_MAP && rows && ok) {
        for (int i = 0; i < n; i++) {
            const double* d = dx + 3 * i;
            double d2 = d[0] * d[0] + d[1] * d[1] + (DIM == 3 ? d[2] * d[2] : 0.0);
            const double w = weight_value<double>(kind, sqrt(d2) * inv_r);
            double u[3];
            basis_offsets<DIM, double>(d, inv_r, recentre ? bcv : nullptr, u);
            double am[M];
            am[0] = 1.0;
            double sdot = y[0];
            sfor<M - 1>([&](auto I) {
                constexpr int p = decltype(I)::value + 1;
                am[p] = am[mono_parent(DIM, p)] * u[mono_var(DIM, p)];
                sdot += am[p] * y[p];
            });
            rows[i] = w * sdot;
        }
    }
    return ok ? 1 : 0;
}

template <int DIM, int DEG>
static int run_mode(int fused, int kind, int n, const double* dx, const double* b, double inv_r,
                    double lambda, double tau, double* mom_out, double* out, int recentre,
                    double* rows) {
    if (fused)
        return run<DIM, DEG, MODE_FUSED>(kind, n, dx, b, inv_r, lambda, tau, mom_out, out, recentre, rows);
    return run<DIM, DEG, MODE_MAP>(kind, n, dx, b, inv_r, lambda, tau, mom_out, out, recentre, rows);
}

extern "C" int hk_mls(int dim, int deg, int fused, int kind, int n, const double* dx,
                      const double* b, double inv_r, double lambda, double tau, double* mom_out,
                      double* out, int recentre, double* rows) {
#define HK_MLS(D, K) return run_mode<D, K>(fused, kind, n, dx, b, inv_r, lambda, tau, mom_out, out, recentre, rows)
    if (dim == 2) {
        if (deg == 0) HK_MLS(2, 0);
        if (deg == 1) HK_MLS(2, 1);
        HK_MLS(2, 2);
    }
    if (deg == 0) HK_MLS(3, 0);
    if (deg == 1) HK_MLS(3, 1);
    HK_MLS(3, 2);
#undef HK_MLS
}

// The mixed path's FP32 arithmetic for one fused target, lane by lane as k_assemble runs it:
// pair i goes to lane i % G (full rounds of G pops, then a tail), scheme 0 = plain sums and a
// shuffle-order FP32 lane reduction (ACC_PLAIN), 1 = blocked compensation with a flush every
// BK_BLOCK full rounds and the TwoSum lane reduction (ACC_BK); basis = re-centred basis
// (c_x, c_y, c_z, 1/s) or null. The moments are then solved in FP64 as k_solve does.
template <int DIM, int DEG>
static int run_f32(int scheme, int kind, int n, const float* dx, const float* b, float inv_r,
                   double lambda, double tau, const float* basis, double* out, int G) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NACC = NM + M;
    if (G < 1 || G > 32 || (G & (G - 1))) return -1;
    float acc[32][NACC], sum[32][NACC], cmp[32][NACC];
    for (int l = 0; l < G; l++)
        for (int i = 0; i < NACC; i++) acc[l][i] = sum[l][i] = cmp[l][i] = 0.f;
    const float* bc = basis;
    const int full = n / G;
    int pops = 0;
    for (int r = 0; r < full; r++) {
        for (int l = 0; l < G; l++) {
            const int i = r * G + l;
            accumulate<DIM, DEG, MODE_FUSED, float, NACC>(acc[l], dx + 3 * i, b[i], kind, inv_r, bc);
        }
        if (scheme == 1 && ++pops == BK_BLOCK) {
            for (int l = 0; l < G; l++) bk_flush<NACC>(acc[l], sum[l], cmp[l]);
            pops = 0;
        }
    }
    for (int l = 0; l < n - full * G; l++) {
        const int i = full * G + l;
        accumulate<DIM, DEG, MODE_FUSED, float, NACC>(acc[l], dx + 3 * i, b[i], kind, inv_r, bc);
    }
    double tot[NACC];
    for (int i = 0; i < NACC; i++) {
        float hi[32], lo[32];
        for (int l = 0; l < G; l++) {
            if (scheme == 1) {
                kahan_add(sum[l][i], cmp[l][i], acc[l][i]);
                hi[l] = sum[l][i];
                lo[l] = -cmp[l][i];
            } else {
                hi[l] = acc[l][i];
                lo[l] = 0.f;
            }
        }
        for (int o = G / 2; o > 0; o >>= 1) {
            float nh[32], nl[32];
            for (int l = 0; l < G; l++) {
                if (scheme == 1) {
                    float s, e;
                    two_sum32(hi[l], hi[l ^ o], s, e);
                    nl[l] = (lo[l] + lo[l ^ o]) + e;
                    nh[l] = s;
                } else {
                    nh[l] = hi[l] + hi[l ^ o];
                    nl[l] = 0.f;
                }
            }
            for (int l = 0; l < G; l++) { hi[l] = nh[l]; lo[l] = nl[l]; }
        }
        tot[i] = (double)hi[0] + (double)lo[0];
    }
    double at[M];
    const double* atp = nullptr;
    if (basis) {
        basis_at_target<DIM, DEG>(make_float4(basis[0], basis[1], basis[2], basis[3]), at);
        atp = at;
    }
    double y[M], c0 = 0.0, amp = 0.0;
    const bool ok = solve_moments<DIM, DEG, MODE_FUSED>(tot, lambda, tau, y, &c0, &amp, atp);
    out[0] = c0;
    out[1] = amp;
    return ok ? 1 : 0;
}

extern "C" int hk_mls_f32(int dim, int deg, int scheme, int kind, int n, const float* dx,
                          const float* b, float inv_r, double lambda, double tau,
                          const float* basis, double* out, int lanes) {
#define HK_F32(D, K) return run_f32<D, K>(scheme, kind, n, dx, b, inv_r, lambda, tau, basis, out, lanes)
    if (dim == 2) {
        if (deg == 1) HK_F32(2, 1);
        HK_F32(2, 2);
    }
    if (deg == 1) HK_F32(3, 1);
    HK_F32(3, 2);
#undef HK_F32
}

// the re-centred basis k_solve derives from target-centred moments
extern "C" void hk_recentre_basis(int dim, const double* mom, float* out) {
    const float4 b = dim == 2 ? recentre_basis<2>(mom) : recentre_basis<3>(mom);
    out[0] = b.x; out[1] = b.y; out[2] = b.z; out[3] = b.w;
}

// The mixed tiers' refined FP32 solve on stored moments: pairs = 0 takes mom_hi as FP32
// sums, 1 as (hi, lo) pairs from mom_hi and mom_lo. at = a_t or null (e_1).
template <int DIM, int DEG, int MODE, typename MT>
static int refined_t(const MT* mt, const double* at, double amp_accept, float* yh, float* yl,
                     double* c0, double* amp) {
    float a = 0.f;
    const int rc = solve_moments_refined<DIM, DEG, MODE, MT>(mt, at, (float)amp_accept, yh, yl,
                                                             c0, &a);
    *amp = (double)a;
    return rc;
}

extern "C" int hk_solve_refined(int dim, int deg, int fused, int pairs, int nacc,
                                const float* mom_hi, const float* mom_lo, const double* at,
                                double amp_accept, float* yh, float* yl, double* c0,
                                double* amp) {
    float m1[64];
    float2 m2[64];
    if (nacc > 64) return -1;
    for (int i = 0; i < nacc; i++) {
        m1[i] = mom_hi[i];
        m2[i] = make_float2(mom_hi[i], mom_lo[i]);
    }
#define HK_R(D, K, MODE)                                                       \
    return pairs ? refined_t<D, K, MODE, float2>(m2, at, amp_accept, yh, yl, c0, amp)      \
                 : refined_t<D, K, MODE, float>(m1, at, amp_accept, yh, yl, c0, amp)
#define HK_RM(D, K)                          \
    if (fused) { HK_R(D, K, MODE_FUSED); }   \
    HK_R(D, K, MODE_MAP)
    if (dim == 2) {
        if (deg == 1) { HK_RM(2, 1); }
        HK_RM(2, 2);
    }
    if (deg == 1) { HK_RM(3, 1); }
    HK_RM(3, 2);
#undef HK_RM
#undef HK_R
}

// the tier-2 basis k_solve derives from moments assembled in the basis b (tier 1's estimate)
extern "C" void hk_recentre_from(int dim, const float* b, const double* mom, float* out) {
    const float4 bb = make_float4(b[0], b[1], b[2], b[3]);
    const float4 r = dim == 2 ? recentre_from<2>(bb, mom) : recentre_from<3>(bb, mom);
    out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
}

extern "C" int hk_mono(int dim, int p, int* e) {
    Exp3 x = mono_exp(dim, p);
    e[0] = x.e[0];
    e[1] = x.e[1];
    e[2] = x.e[2];
    return mono_count(dim, 8);
}

extern "C" int hk_mono_prod(int dim, int k, int l) { return mono_prod(dim, k, l); }

extern "C" double hk_weight(int kind, double q) { return weight_value<double>(kind, q); }

// the compile-time pairing of the FP32 moment terms (two-lane FP32 instructions)
template <int DIM, int MDEG>
static int pair_plan(int* partner, int* first, int* packed) {
    constexpr PairPlan<DIM, MDEG> P = PairPlanOf<DIM, MDEG>::v;
    for (int p = 0; p < P.N; ++p) {
        partner[p] = P.partner[p];
        first[p] = P.first[p] ? 1 : 0;
        packed[p] = P.packed[p] ? 1 : 0;
    }
    return P.N;
}

extern "C" int hk_pair_plan(int dim, int mdeg, int* partner, int* first, int* packed) {
    if (dim == 2 && mdeg == 2) return pair_plan<2, 2>(partner, first, packed);
    if (dim == 2 && mdeg == 4) return pair_plan<2, 4>(partner, first, packed);
    if (dim == 3 && mdeg == 2) return pair_plan<3, 2>(partner, first, packed);
    if (dim == 3 && mdeg == 4) return pair_plan<3, 4>(partner, first, packed);
    return -1;
}
