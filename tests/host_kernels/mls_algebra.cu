// Host-compiled harness for the CPU tests: exposes the library's per-target MLS algebra
// (the moment accumulation and the guarded LDL^T solve from mls_kernels.cuh, compiled for
// the host with T = double) so its arithmetic can be checked against numpy without a GPU.
#include "mls_kernels.cuh"

using namespace pcms;

template <int DIM, int DEG, int MODE>
static int run(int kind, int n, const double* dx, const double* b, double inv_r, double lambda,
               double tau, double* mom_out, double* out) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NACC = MODE == MODE_FUSED ? NM + M : NM;
    double acc[NACC], cmp[NACC];
    for (int i = 0; i < NACC; i++) acc[i] = cmp[i] = 0.0;
    for (int i = 0; i < n; i++)
        accumulate<DIM, DEG, MODE, double, NACC>(acc, cmp, dx + 3 * i, b ? b[i] : 0.0, kind, inv_r);
    for (int i = 0; i < NACC; i++) mom_out[i] = acc[i];
    double y[M], c0 = 0.0, amp = 0.0;
    const bool ok = solve_moments<DIM, DEG, MODE>(acc, lambda, tau, y, &c0, &amp);
    if (MODE == MODE_FUSED) out[0] = c0;
    else
        for (int k = 0; k < M; k++) out[k] = y[k];
    out[M] = amp;
    return ok ? 1 : 0;
}

template <int DIM, int DEG>
static int run_mode(int fused, int kind, int n, const double* dx, const double* b, double inv_r,
                    double lambda, double tau, double* mom_out, double* out) {
    if (fused) return run<DIM, DEG, MODE_FUSED>(kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
    return run<DIM, DEG, MODE_MAP>(kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
}

extern "C" int hk_mls(int dim, int deg, int fused, int kind, int n, const double* dx,
                      const double* b, double inv_r, double lambda, double tau, double* mom_out,
                      double* out) {
    if (dim == 2) {
        if (deg == 0) return run_mode<2, 0>(fused, kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
        if (deg == 1) return run_mode<2, 1>(fused, kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
        return run_mode<2, 2>(fused, kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
    }
    if (deg == 0) return run_mode<3, 0>(fused, kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
    if (deg == 1) return run_mode<3, 1>(fused, kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
    return run_mode<3, 2>(fused, kind, n, dx, b, inv_r, lambda, tau, mom_out, out);
}

// FP32 accumulation (plain or compensated) of the same per-pair algebra, reduced in FP64,
// then the FP64 solve: the arithmetic of precision tiers 1 and 2 of the mixed path
template <int DIM, int DEG, bool COMP>
static int run_f32(int kind, int n, const float* dx, const float* b, float inv_r, double lambda,
                   double tau, double* out, int lanes) {
    constexpr int NM = mono_count(DIM, 2 * DEG);
    constexpr int M = mono_count(DIM, DEG);
    constexpr int NACC = NM + M;
    double tot[NACC];
    for (int i = 0; i < NACC; i++) tot[i] = 0.0;
    for (int l = 0; l < lanes; l++) {
        float acc[NACC], cmp[NACC];
        for (int i = 0; i < NACC; i++) acc[i] = cmp[i] = 0.f;
        for (int i = l; i < n; i += lanes)
            accumulate<DIM, DEG, MODE_FUSED, float, NACC, COMP>(acc, cmp, dx + 3 * i, b[i], kind, inv_r);
        for (int i = 0; i < NACC; i++) tot[i] += (double)acc[i] - (double)cmp[i];
    }
    double y[M], c0 = 0.0, amp = 0.0;
    const bool ok = solve_moments<DIM, DEG, MODE_FUSED>(tot, lambda, tau, y, &c0, &amp);
    out[0] = c0;
    out[1] = amp;
    return ok ? 1 : 0;
}

extern "C" int hk_mls_f32(int dim, int deg, int comp, int kind, int n, const float* dx,
                          const float* b, float inv_r, double lambda, double tau, double* out,
                          int lanes) {
#define HK_F32(D, K)                                                                         \
    return comp ? run_f32<D, K, true>(kind, n, dx, b, inv_r, lambda, tau, out, lanes)        \
                : run_f32<D, K, false>(kind, n, dx, b, inv_r, lambda, tau, out, lanes)
    if (dim == 2) {
        if (deg == 1) HK_F32(2, 1);
        HK_F32(2, 2);
    }
    if (deg == 1) HK_F32(3, 1);
    HK_F32(3, 2);
#undef HK_F32
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
