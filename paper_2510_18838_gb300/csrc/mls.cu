// mls.cu -- host orchestration of the MLS transfer (Sec. 3.2.1): grid build, neighbour
// count, operator assembly/solve/shape, one-shot transfer, apply and export.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mls_dispatch.cuh"

namespace pcms {

namespace {

constexpr int64_t MAX_CELLS = int64_t(1) << 24;
constexpr double TAU_FP64 = 1e-14;   // (1e-7)^2: column-angle rank test of the definition
constexpr double TAU_MIXED = 1e-5;   // plain-FP32 pivots below this go to the next tier
constexpr double TAU_BK = 1e-7;      // blocked-compensated pivots below this go on (noise ~1e-8)

// stored moment type of an assembly
int mom_kind(bool mixed, int acc) {
    return !mixed ? MOM_F64 : (acc == ACC_BK ? MOM_F32PAIR : MOM_F32);
}
size_t mom_elem_bytes(int kind) { return kind == MOM_F32 ? sizeof(float) : sizeof(double); }

int asm_blocks(int64_t nwork, int G) {
    int64_t groups_per_block = 8 * (32 / G);
    int64_t need = (nwork + groups_per_block - 1) / groups_per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 16));
}

int thread_blocks(int64_t n, int threads) {
    int64_t need = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 32));
}

// k_rows64_apply for the listed flag-2 targets (count on the device)
void rows64_apply_any(int dim, int deg, int G, const ShapeArgs& sh, const int32_t* list,
                      const int32_t* n, int64_t nmax, cudaStream_t s) {
    if (nmax <= 0) return;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((nmax * G + 255) / 256, (int64_t)num_sms() * 8));
#define PCMS_R64(D, K, GG) k_rows64_apply<D, K, GG><<<blocks, 256, 0, s>>>(sh, list, n)
    if (dim == 2) {
        if (G == 32) { if (deg == 0) PCMS_R64(2, 0, 32); else if (deg == 1) PCMS_R64(2, 1, 32); else PCMS_R64(2, 2, 32); }
        else { if (deg == 0) PCMS_R64(2, 0, 8); else if (deg == 1) PCMS_R64(2, 1, 8); else PCMS_R64(2, 2, 8); }
    } else {
        if (G == 32) { if (deg == 0) PCMS_R64(3, 0, 32); else if (deg == 1) PCMS_R64(3, 1, 32); else PCMS_R64(3, 2, 32); }
        else { if (deg == 0) PCMS_R64(3, 0, 8); else if (deg == 1) PCMS_R64(3, 1, 8); else PCMS_R64(3, 2, 8); }
    }
#undef PCMS_R64
    PCMS_LAUNCH_CHECK("k_rows64_apply");
}

// Lanes per target, the first pass's accumulation and the grid's cell edge, from the expected
// neighbour count (ns * ball volume / box volume).
//  - 32 lanes from 160 neighbours on, else 8; operators from 320 on (the lockstep 8-lane
//    walk stages 384 columns per target: on the serving stream, 8 lanes up to 320 neighbours
//    cut the step from 744 to 711 ms).
//  - Blocked compensation (mixed path) from 1000 on, where plain FP32 sums over n / 32 pairs
//    per lane stop meeting the error bound for ordinary targets; below that plain sums pass
//    for almost every target and the blocked form would only cost registers.
//  - Cell edge r/3 in 2D, r/2 in 3D; r/6 in 2D from 1000 neighbours on. Smaller cells trim
//    candidate rows closer to the ball at the price of more rows per target; measured on the
//    4M 2D and 8M 3D transfers, r/3 is 5% faster in 2D and 6% slower in 3D than r/2, and with
//    thousands of candidates per row the rows of r/6 cells cost little beside the candidates
//    they save.
// An entry of the tuning table (pcms_tune_set: lanes and cell divisor measured fastest for
// this dimension, degree, precision, mode and count bucket) replaces the lanes and the cell
// edge; the accumulation stays the precision rule's (blocked compensation needs 32 lanes).
struct AsmPlan {
    int G;
    int acc;
    double mean;   // expected neighbours per target
    double cell;   // grid cell edge
    int xs;        // x cells per cell edge (choose_xs)
    bool tuned;
};
AsmPlan choose_plan(int dim, int deg, int mode, int64_t ns, double radius, const double* lo,
                    const double* hi, bool mixed) {
    double vol = 1.0;
    for (int d = 0; d < dim; d++) vol *= std::max(hi[d] - lo[d], radius);
    double ball = dim == 2 ? M_PI * radius * radius : 4.0 / 3.0 * M_PI * radius * radius * radius;
    double mean = (double)ns * ball / vol;
    AsmPlan p;
    p.mean = mean;
    p.G = mean >= (mode == MODE_MAP ? 320.0 : 160.0) ? 32 : 8;
    double div = dim == 2 ? (mean >= 1000.0 ? 6.0 : 3.0) : 2.0;
    p.tuned = false;
    TuneEntry e;
    if (mode != MODE_COUNT && tune_lookup(dim, deg, mixed, mode, tune_bucket(mean), &e)) {
        p.G = e.lanes;
        div = e.cell_div;
        p.tuned = true;
    }
    const bool bk = mixed && mean >= 1000.0;
    if (bk) p.G = 32;
    p.acc = bk ? ACC_BK : ACC_PLAIN;
    p.cell = radius / div;
    p.xs = choose_xs(dim, lo, hi, p.cell, MAX_CELLS, ns);
    return p;
}

// out: [0] underdetermined, [1] ill-conditioned, [2] max count, [3] max doublings,
//      [4] sum of counts (the operator's nonzeros)
__global__ void __launch_bounds__(256) k_stats(const int8_t* status, const int32_t* counts,
                                               const int32_t* kexp, int64_t n,
                                               unsigned long long* out) {
    unsigned long long under = 0, ill = 0, mc = 0, mk = 0, sc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int8_t st = status[i];
        under += st == PCMS_TARGET_UNDERDETERMINED;
        ill += st == PCMS_TARGET_ILL_CONDITIONED;
        mc = max(mc, (unsigned long long)counts[i]);
        mk = max(mk, (unsigned long long)kexp[i]);
        sc += (unsigned long long)counts[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        under += __shfl_xor_sync(0xffffffffu, under, o);
        ill += __shfl_xor_sync(0xffffffffu, ill, o);
        mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
    }
    // one set of atomics per block: per-warp atomics on five addresses serialise in L2
    __shared__ unsigned long long sh[8][5];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[w][0] = under;
        sh[w][1] = ill;
        sh[w][2] = mc;
        sh[w][3] = mk;
        sh[w][4] = sc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < (int)(blockDim.x >> 5); j++) {
            under += sh[j][0];
            ill += sh[j][1];
            mc = max(mc, sh[j][2]);
            mk = max(mk, sh[j][3]);
            sc += sh[j][4];
        }
        atomicAdd(&out[0], under);
        atomicAdd(&out[1], ill);
        atomicMax(&out[2], mc);
        atomicMax(&out[3], mk);
        atomicAdd(&out[4], sc);
    }
}

int stats_blocks(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 2 * (int64_t)num_sms()));
}

template <typename T>
__global__ void k_permute_field(const T* __restrict__ f, const int32_t* __restrict__ inv,
                                int64_t n, T* __restrict__ fs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        fs[inv[i]] = f[i];
}

// sum of the neighbour counts of the targets on a list (tracing only: pairs per tier)
__global__ void k_list_pairs(const int32_t* __restrict__ list, const int32_t* __restrict__ n_list,
                             const int32_t* __restrict__ counts, unsigned long long* out) {
    unsigned long long s = 0;
    const int64_t n = *n_list;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)counts[list[i]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

void trace_list_pairs(const char* name, const int32_t* list, const int32_t* n_list,
                      const int32_t* counts, int64_t n, cudaStream_t s) {
    if (!trace_timing() || n <= 0) return;
    DBuf acc(sizeof(unsigned long long), s);
    PCMS_CU(cudaMemsetAsync(acc.p, 0, acc.bytes, s));
    k_list_pairs<<<thread_blocks(n, 256), 256, 0, s>>>(list, n_list, counts,
                                                       acc.as<unsigned long long>());
    PCMS_LAUNCH_CHECK("k_list_pairs");
    unsigned long long h = 0;
    PCMS_CU(cudaMemcpyAsync(&h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    trace_count(name, (int64_t)h);
}

struct BoxResult {
    double lo[3], hi[3];
};

// Bounding box of the sources and a finiteness check of sources and targets (one sync),
// or the caller's box.
BoxResult source_box(int dim, const double* src, int64_t ns, const double* tgt, int64_t nt,
                     const pcms_map_opts& o, cudaStream_t s) {
    BoxResult b;
    if (o.domain_known) {
        for (int d = 0; d < 3; d++) { b.lo[d] = o.lo[d]; b.hi[d] = o.hi[d]; }
        return b;
    }
    // per-block partial boxes of both point sets, one copy back, combined here
    const int bs = bbox_blocks(ns), bt = bbox_blocks(nt);
    DBuf part(sizeof(double) * 8 * (bs + bt), s);
    launch_bbox_partials(dim, src, ns, part.as<double>(), s);
    launch_bbox_partials(dim, tgt, nt, part.as<double>() + 8 * bs, s);
    std::vector<double> hp(8 * (size_t)(bs + bt));
    if (ns > 0)
        PCMS_CU(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * 8 * bs, cudaMemcpyDeviceToHost, s));
    if (nt > 0)
        PCMS_CU(cudaMemcpyAsync(hp.data() + 8 * bs, part.as<double>() + 8 * bs,
                                sizeof(double) * 8 * bt, cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    double slo[3], shi[3], tlo[3], thi[3];
    uint64_t sbad = 0, tbad = 0;
    bbox_combine(hp.data(), ns, slo, shi, &sbad);
    bbox_combine(hp.data() + 8 * bs, nt, tlo, thi, &tbad);
    if (sbad || tbad)
        fail(PCMS_ERR_INVALID_ARG, "non-finite point coordinate (" + std::to_string(sbad) +
                                       " in sources, " + std::to_string(tbad) + " in targets)");
    for (int d = 0; d < 3; d++) {
        b.lo[d] = (d < dim && ns > 0) ? slo[d] : 0.0;
        b.hi[d] = (d < dim && ns > 0) ? shi[d] : 0.0;
    }
    return b;
}

AsmArgs base_args(const Grid& g, const SortedPoints& S, const SortedPoints& Tp,
                  const MlsParams& P) {
    AsmArgs a{};
    a.g = g;
    a.ns = S.n;
    a.nt = Tp.n;
    a.cell_start = S.cell_start.as<int32_t>();
    a.sx64 = S.x64.as<double>();
    a.hl0 = S.hl0.as<float4>();
    a.hl1 = S.hl1.as<float2>();
    a.tx64 = Tp.x64.as<double>();
    a.thl0 = Tp.hl0.as<float4>();
    a.thl1 = Tp.hl1.as<float2>();
    a.tcell = Tp.cell.as<int4>();
    a.tfrac = Tp.frac.as<float4>();
    a.lv = make_radius_levels(P.radius, g.inv_h);
    a.radius = P.radius;
    a.weight = (int)P.weight;
    a.need = P.need;
    return a;
}

// Tier-1 basis estimates (estimate_basis): blocked-compensated mixed plans at lambda = 0
// and degree >= 1 assemble targets whose estimated neighbour centroid lies more than
// RECENTRE_MIN radii away in that re-centred basis, so that they pass in tier 1 instead of
// being walked again in tier 2. Returns the buffers (per-cell means, per-target basis).
constexpr float RECENTRE_MIN = 0.5f;

struct BasisEstimate {
    DBuf pyr, basis;
    int levels = 0;
    int64_t off[PYR_MAX] = {};
    void enable(bool mixed, const AsmPlan& plan, const MlsParams& P, const Grid& g,
                const SortedPoints& S, int64_t nt, cudaStream_t s) {
        if (!(mixed && plan.acc == ACC_BK && P.degree >= 1 && P.lambda == 0.0) || nt <= 0 ||
            g.ncell <= 0)
            return;
        levels = pyramid_levels(g);
        pyr.alloc(sizeof(float4) * pyramid_size(g, levels, off), s);
        basis.alloc(sizeof(float4) * nt, s);
        cell_pyramid(g, S, levels, off, pyr.as<float4>(), s);
    }
    void apply(AsmArgs& a) const {
        if (!basis.p) return;
        a.cpyr = pyr.as<float4>();
        for (int j = 0; j < PYR_MAX; j++) a.pyr_off[j] = off[j];
        a.pyr_levels = levels;
        a.basis_out = basis.as<float4>();
        a.recentre_min2 = RECENTRE_MIN * RECENTRE_MIN;
    }
    void apply(SolveArgs& sa) const { sa.basis_in = basis.p ? basis.as<float4>() : nullptr; }
};

int accp(int dim, int deg, int mode) {
    int nm = mono_count(dim, 2 * deg), m = mono_count(dim, deg);
    int nacc = mode == MODE_FUSED ? nm + m : nm;
    return round_up4(nacc);
}

// Solve the tier-1 systems already assembled in sa.mom, then re-assemble and solve the
// targets the solve hands on: tier 2 (blocked-compensated FP32, 32 lanes, re-centred basis
// when lambda = 0) and tier 3 (FP64). `a` holds the assembly arguments of tier 1
// (mode-specific fields set). The mixed path syncs to size the tier-2/3 work; the FP64 path
// has a single tier. rc: MAP only, per-target basis of re-centred operator rows.
void solve_tiers(int dim, int deg, int mode, bool mixed, AsmPlan plan, const AsmArgs& a,
                 SolveArgs sa, int64_t nt, float4* rc, cudaStream_t s) {
    const int np = accp(dim, deg, mode);
    const int G = plan.G;
    const int mk1 = mom_kind(mixed, plan.acc);
    DBuf lists(sizeof(int32_t) * (3 * nt + 4), s);
    int32_t* list2 = lists.as<int32_t>();
    int32_t* list3 = list2 + nt;
    int32_t* fb = list3 + nt;   // the refined solve's declined work items (per mixed pass)
    int32_t* n2 = fb + nt;
    int32_t* n3 = n2 + 1;
    int32_t* n_rc = n2 + 2;
    int32_t* n_fb = n2 + 3;
    DBuf basis2(sizeof(float4) * nt, s);
    PCMS_CU(cudaMemsetAsync(n2, 0, 4 * sizeof(int32_t), s));
    sa.fb_list = fb;
    sa.n_fb = n_fb;
    sa.list2 = list2;
    sa.n2 = n2;
    sa.list3 = list3;
    sa.n3 = n3;
    sa.tier = mixed ? 1 : 3;
    sa.group = G;
    sa.acc = mk1 == MOM_F32PAIR ? ACC_BK : ACC_PLAIN;
    sa.recentre = mixed && deg >= 1 && sa.lambda == 0.0;
    sa.refine64 = !mixed && deg >= 1 && sa.lambda == 0.0;
    sa.tau = !mixed ? TAU_FP64 : (sa.acc == ACC_BK ? TAU_BK : TAU_MIXED);
    // sa.basis_in: the caller's tier-1 basis estimates (BasisEstimate), or null
    sa.n_recentred = sa.basis_in ? n_rc : nullptr;
    sa.basis2 = basis2.as<float4>();
    sa.rc = rc;
    solve_any(dim, deg, mode, mk1, sa, thread_blocks(nt, 128), s);
    if (!mixed) {
        if (!sa.refine64) return;
        // FP64 refine pass: the listed targets again, in their re-centred bases
        int32_t n_ref = 0;
        PCMS_CU(cudaMemcpyAsync(&n_ref, n2, sizeof(n_ref), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
        trace_count("mls_fp64_refine_targets", n_ref);
        if (n_ref == 0) return;
        DBuf mom4(sizeof(double) * np * n_ref, s);
        AsmArgs a4 = a;
        a4.cpyr = nullptr;
        a4.basis_out = nullptr;
        a4.list = list2;
        a4.n_list = n2;
        a4.mom = mom4.p;
        a4.basis = basis2.as<float4>();
        if (mode == MODE_FUSED) {
            a4.kexp_in = a.kexp_out ? a.kexp_out : a.kexp_in;
            a4.kexp_out = nullptr;
        } else {
            a4.cols = nullptr;   // the operator's columns are already written
        }
        // the FP64 path's fields are double (fd)
        assemble_any(dim, deg, false, mode, G, ACC_PLAIN, true, a4, asm_blocks(n_ref, G), s);
        SolveArgs s4 = sa;
        s4.n_recentred = nullptr;
        s4.list = list2;
        s4.n_list = n2;
        s4.mom = mom4.p;
        s4.tier = 4;
        s4.acc = ACC_PLAIN;
        s4.tau = TAU_FP64;
        s4.refine64 = 0;
        s4.basis_in = basis2.as<float4>();
        s4.basis2 = nullptr;
        solve_any(dim, deg, mode, MOM_F64, s4, thread_blocks(n_ref, 128), s);
        return;
    }
    int32_t cnt[4] = {0, 0, 0, 0};
    PCMS_CU(cudaMemcpyAsync(cnt, n2, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    trace_count("mls_tier1_fp64_solves", cnt[3]);
    trace_count("mls_tier1_targets", nt - cnt[0] - cnt[1]);
    trace_count("mls_tier1_recentred_solves", cnt[2]);
    trace_count("mls_tier2_targets", cnt[0]);
    trace_list_pairs(mode == MODE_FUSED ? "mls_fused_tier2_pairs" : "mls_map_tier2_pairs", list2,
                     n2, sa.counts, cnt[0], s);
    if (cnt[0] > 0) {
        DBuf mom2(sizeof(float2) * np * cnt[0], s);
        AsmArgs a2 = a;
        a2.cpyr = nullptr;
        a2.basis_out = nullptr;
        a2.list = list2;
        a2.n_list = n2;
        a2.mom = mom2.p;
        a2.basis = basis2.as<float4>();
        if (mode == MODE_FUSED) {
            a2.kexp_in = a.kexp_out ? a.kexp_out : a.kexp_in;
            a2.kexp_out = nullptr;
        } else {
            a2.cols = nullptr;   // the operator's columns are already written
        }
        // tier 2 keeps tier 1's lanes per target: its targets are mostly small, badly
        // conditioned neighbourhoods, which 32 lanes would spend on reductions
        assemble_any(dim, deg, true, mode, G, ACC_BK, false, a2, asm_blocks(cnt[0], G), s);
        SolveArgs s2 = sa;
        s2.n_recentred = nullptr;
        PCMS_CU(cudaMemsetAsync(n_fb, 0, sizeof(int32_t), s));   // tier 2's own declined items
        s2.list = list2;
        s2.n_list = n2;
        s2.mom = mom2.p;
        s2.tier = 2;
        s2.acc = ACC_BK;
        s2.tau = TAU_BK;
        s2.basis_in = basis2.as<float4>();
        s2.basis2 = nullptr;
        solve_any(dim, deg, mode, MOM_F32PAIR, s2, thread_blocks(cnt[0], 128), s);
        PCMS_CU(cudaMemcpyAsync(&cnt[1], n3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
    }
    trace_count("mls_tier3_targets", cnt[1]);
    trace_list_pairs(mode == MODE_FUSED ? "mls_fused_tier3_pairs" : "mls_map_tier3_pairs", list3,
                     n3, sa.counts, cnt[1], s);
    if (cnt[1] > 0) {
        DBuf mom3(sizeof(double) * np * cnt[1], s);
        AsmArgs a3 = a;
        a3.cpyr = nullptr;
        a3.basis_out = nullptr;
        a3.list = list3;
        a3.n_list = n3;
        a3.mom = mom3.p;
        a3.basis = nullptr;
        if (mode == MODE_FUSED) {
            a3.kexp_in = a.kexp_out ? a.kexp_out : a.kexp_in;
            a3.kexp_out = nullptr;
        } else {
            a3.cols = nullptr;
        }
        assemble_any(dim, deg, false, mode, G, ACC_PLAIN, false, a3, asm_blocks(cnt[1], G), s);
        SolveArgs s3 = sa;
        s3.n_recentred = nullptr;
        s3.list = list3;
        s3.n_list = n3;
        s3.mom = mom3.p;
        s3.tier = 3;
        s3.acc = ACC_PLAIN;
        s3.tau = TAU_FP64;
        s3.basis_in = nullptr;
        s3.basis2 = nullptr;
        solve_any(dim, deg, mode, MOM_F64, s3, thread_blocks(cnt[1], 128), s);
    }
}

__global__ void k_max_i32(const int32_t* __restrict__ v, int64_t n, unsigned long long* out) {
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)max(v[i], 0));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// Global reading of the minimum-count rule (Sec. 3.2.1): one count pass with per-target
// growth gives every target's doublings k_t. A target's count only grows with the radius,
// so the fewest shared doublings after which no target is short is K = max_t k_t. The
// request then runs at the fixed radius radius * 2^K (exact in FP64), and K is added to
// the exponents it reports.
MlsParams settle_growth(const MlsParams& P, const double* src, int64_t ns, const double* tgt,
                        int64_t nt, const pcms_map_opts& o, cudaStream_t s) {
    if (P.need == 0 || P.growth != PCMS_GROWTH_GLOBAL || nt == 0) return P;
    const int dim = P.dim;
    const bool mixed = P.prec == PCMS_MIXED;
    BoxResult b = source_box(dim, src, ns, tgt, nt, o, s);
    const AsmPlan cplan = choose_plan(dim, 0, MODE_COUNT, ns, P.radius, b.lo, b.hi, mixed);
    Grid g = make_grid(dim, b.lo, b.hi, cplan.cell, MAX_CELLS, cplan.xs);
    SortedPoints S, Tp;
    sort_points(g, src, ns, true, mixed, S, s);
    sort_points(g, tgt, nt, false, mixed, Tp, s, true);
    const int G = cplan.G;
    DBuf c(sizeof(int32_t) * nt, s);
    DBuf k(sizeof(int32_t) * nt, s);
    DBuf mx(sizeof(unsigned long long), s);
    PCMS_CU(cudaMemsetAsync(mx.p, 0, mx.bytes, s));
    AsmArgs a = base_args(g, S, Tp, P);
    a.counts = c.as<int32_t>();
    a.kexp_out = k.as<int32_t>();
    assemble_any(dim, 0, mixed, MODE_COUNT, G, ACC_PLAIN, false, a, asm_blocks(nt, G), s);
    {
        PCMS_TRACE("mls_global_doublings", s);
        k_max_i32<<<thread_blocks(nt, 256), 256, 0, s>>>(k.as<int32_t>(), nt,
                                                        mx.as<unsigned long long>());
    }
    PCMS_LAUNCH_CHECK("k_max_i32");
    unsigned long long K = 0;
    PCMS_CU(cudaMemcpyAsync(&K, mx.p, sizeof(K), cudaMemcpyDeviceToHost, s));
    PCMS_CU(cudaStreamSynchronize(s));
    MlsParams Q = P;
    Q.radius = std::ldexp(P.radius, (int)K);
    Q.need = 0;
    Q.kbase = (int)K;
    return Q;
}

}  // namespace

MlsParams make_mls_params(int dim, int degree, double radius, const pcms_map_opts& o) {
    MlsParams P;
    P.dim = dim;
    P.degree = degree;
    P.m = mono_count(dim, degree);
    P.prec = o.precision;
    P.weight = o.weight;
    P.radius = radius;
    P.lambda = o.lambda;
    P.min_neighbors = o.min_neighbors;
    P.need = o.min_neighbors > 0 ? std::max(o.min_neighbors, P.m) : 0;
    P.growth = o.growth;
    P.kbase = 0;
    return P;
}

int64_t estimate_mls_bytes(const MlsParams& P, int64_t ns, int64_t nt, int nf, bool keep_map) {
    const int d = P.dim;
    const bool mixed = P.prec == PCMS_MIXED;
    // volume of the d-ball of radius r: pi^(d/2) r^d / Gamma(d/2 + 1)
    const double ball = std::pow(M_PI, 0.5 * d) * std::pow(P.radius, d) / std::tgamma(0.5 * d + 1.0);
    double k = std::max((double)P.m, std::max((double)P.need, (double)ns * ball));
    k = std::min(k, (double)std::max<int64_t>(ns, 1));
    const double elem = mixed ? 4.0 : 8.0;
    const int np = round_up4(mono_count(d, 2 * P.degree) + P.m);
    double b = 0;
    b += ns * (4.0 + 4.0 + 8.0 * d + (mixed ? 24.0 : 0.0) + 12.0);   // sorted sources + sort scratch
    b += nt * (4.0 + 4.0 + 8.0 * d + 12.0);                          // sorted targets + scratch
    b += nt * (4.0 + 4.0 + 1.0 + 8.0 + 4.0);                         // counts, kexp, status, offsets, redo
    b += nt * (np * 8.0 + P.m * 8.0);                                // moments, y
    b += nt * 33.0;                                                  // re-centred bases, row flags
    const double nnz = 1.3 * k * nt;
    if (keep_map || nf > 2) b += nnz * (4.0 + elem);                 // operator
    int fw = 1;                                                      // fields padded to the
    while (fw * (mixed ? 4 : 2) < nf) fw <<= 1;                      // apply's vector width
    const double fp = nf <= 1 ? 1.0 : (double)fw * (mixed ? 4 : 2);
    b += (double)(ns + nt) * fp * elem * 2.0;                        // apply/permute scratch
    b += (mixed ? 26.0 : 4.0) * std::min<double>((double)(int64_t(1) << 24), 2.0 * ns + 64.0);
    // cell starts (and, mixed, the cell-sum pyramid of the tier-1 basis estimates)
    if (mixed) b += nt * 16.0;                                       // estimated bases
    return (int64_t)(1.15 * b) + (int64_t(1) << 20);
}

int64_t MapImpl::device_bytes() const {
    return (int64_t)(src.cell_start.bytes + src.perm.bytes + src.inv.bytes + src.x64.bytes +
                     src.hl0.bytes + src.hl1.bytes + tgt.perm.bytes + tgt.inv.bytes +
                     tgt.x64.bytes + counts.bytes + kexp.bytes + status.bytes + offsets.bytes +
                     cols.bytes + vals.bytes + qr_list.bytes + qr_cols.bytes + qr_vals.bytes +
                     qr_cnt.bytes);
}

// ------------------------------------------------------------------------------------
// create map
// ------------------------------------------------------------------------------------
void mls_create_map(MapImpl& M, const double* src, const double* tgt, const pcms_map_opts& o,
                    const FusedApply* fused) {
    if (fused && (M.P.dim >= 4 || M.P.prec != PCMS_MIXED))
        fail(PCMS_ERR_INVALID_ARG, "internal: rows applied as evaluated need a mixed 2D/3D map");
    if (M.P.dim >= 4) return mls_nd_create_map(M, src, tgt);
    cudaStream_t s = M.stream;
    M.P = settle_growth(M.P, src, M.ns, tgt, M.nt, o, s);
    const MlsParams& P = M.P;
    const int dim = P.dim, deg = P.degree, m = P.m;
    const bool mixed = P.prec == PCMS_MIXED;
    const int64_t ns = M.ns, nt = M.nt;
    BoxResult b = source_box(dim, src, ns, tgt, nt, o, s);
    const AsmPlan plan = choose_plan(dim, deg, MODE_MAP, ns, P.radius, b.lo, b.hi, mixed);
    M.g = make_grid(dim, b.lo, b.hi, plan.cell, MAX_CELLS, plan.xs);
    sort_points(M.g, src, ns, true, mixed, M.src, s);
    sort_points(M.g, tgt, nt, false, mixed, M.tgt, s, true);
    const int G = plan.G;

    M.counts.alloc(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    M.kexp.alloc(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    M.status.alloc(sizeof(int8_t) * std::max<int64_t>(nt, 1), s);
    M.offsets.alloc(sizeof(int64_t) * (nt + 1), s);
    DBuf err(sizeof(unsigned) * 4, s);
    PCMS_CU(cudaMemsetAsync(err.p, 0, err.bytes, s));

    AsmArgs a = base_args(M.g, M.src, M.tgt, P);
    a.err = err.as<unsigned>();
    a.counts = M.counts.as<int32_t>();
    a.kexp_out = M.kexp.as<int32_t>();
    BasisEstimate bases;   // used by the row assembly (MODE_MAP), not by the count pass
    // Rows. With a fixed radius the assembly stages each target's columns, reserves its row
    // with one atomic add and writes it (one pass; the rare rows that do not fit are walked
    // again). When the radius may grow, a count pass finds the doublings and the row sizes.
    const bool one_pass = P.need == 0;
    int64_t nnz = 0;
    if (!one_pass) {
        if (nt > 0)
            assemble_any(dim, 0, mixed, MODE_COUNT, G, ACC_PLAIN, false, a, asm_blocks(nt, G), s);
        exclusive_scan<int64_t>(M.counts.as<int32_t>(), M.offsets.as<int64_t>(), nt, s);
        PCMS_CU(cudaMemcpyAsync(&nnz, M.offsets.as<int64_t>() + nt, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
        M.cols.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1), s);
    }

    if (nt > 0) {
        const int np = accp(dim, deg, MODE_MAP);
        const size_t melem = mom_elem_bytes(mom_kind(mixed, plan.acc));
        DBuf mom(melem * np * nt, s);
        DBuf y(sizeof(double) * m * nt, s);
        DBuf yf(mixed ? sizeof(float2) * m * nt : 0, s);
        DBuf flags(sizeof(int8_t) * nt, s);
        DBuf rc(sizeof(float4) * nt, s);
        a.offsets = M.offsets.as<int64_t>();
        a.mom = mom.p;
        bases.enable(mixed, plan, P, M.g, M.src, nt, s);
        bases.apply(a);
        if (one_pass) {
            const int64_t est = (int64_t)(1.3 * std::min(plan.mean, (double)ns) * (double)nt) + 4096;
            M.cols.alloc(sizeof(int32_t) * est, s);
            DBuf ctl(sizeof(unsigned long long) + sizeof(int32_t) * (nt + 2), s);
            auto* ctr = ctl.as<unsigned long long>();
            int32_t* n_redo = (int32_t*)(ctr + 1);
            int32_t* redo = n_redo + 2;
            PCMS_CU(cudaMemsetAsync(ctl.p, 0, sizeof(unsigned long long) + 2 * sizeof(int32_t), s));
            a.one_pass = 1;
            a.nnz_ctr = ctr;
            a.cols_cap = est;
            a.redo = redo;
            a.n_redo = n_redo;
            a.cols = M.cols.as<int32_t>();
            a.kexp_in = nullptr;
            a.kexp_out = M.kexp.as<int32_t>();
            assemble_any(dim, deg, mixed, MODE_MAP, G, plan.acc, false, a, asm_blocks(nt, G), s);
            unsigned long long hctr = 0;
            int32_t hredo = 0;
            PCMS_CU(cudaMemcpyAsync(&hctr, ctr, sizeof(hctr), cudaMemcpyDeviceToHost, s));
            PCMS_CU(cudaMemcpyAsync(&hredo, n_redo, sizeof(hredo), cudaMemcpyDeviceToHost, s));
            PCMS_CU(cudaStreamSynchronize(s));
            nnz = (int64_t)hctr;
            if (nnz > est) {   // rows reserved past the buffer: grow it, keep what was written
                DBuf grown(sizeof(int32_t) * nnz, s);
                PCMS_CU(cudaMemcpyAsync(grown.p, M.cols.p, sizeof(int32_t) * est,
                                        cudaMemcpyDeviceToDevice, s));
                M.cols = std::move(grown);
            }
            trace_count("mls_map_rows_walked_again", hredo);
            a.one_pass = 0;
            a.kexp_in = M.kexp.as<int32_t>();
            a.kexp_out = nullptr;
            if (hredo > 0) {   // rows that did not fit: walk again, writing at the reserved start
                DBuf mom2(melem * np * hredo, s);
                AsmArgs a2 = a;   // columns only: the first pass's moments and bases stand
                a2.cpyr = nullptr;
                a2.basis_out = nullptr;
                a2.list = redo;
                a2.n_list = n_redo;
                a2.mom = mom2.p;
                a2.cols = M.cols.as<int32_t>();
                assemble_any(dim, deg, mixed, MODE_MAP, G, plan.acc, false, a2,
                             asm_blocks(hredo, G), s);
            }
        } else {
            a.kexp_in = M.kexp.as<int32_t>();
            a.kexp_out = nullptr;
            a.cols = M.cols.as<int32_t>();
            assemble_any(dim, deg, mixed, MODE_MAP, G, plan.acc, false, a, asm_blocks(nt, G), s);
        }
        M.nnz = nnz;
        if (!fused)
            M.vals.alloc((mixed ? sizeof(float) : sizeof(double)) * std::max<int64_t>(nnz, 1), s);

        DBuf qrl(sizeof(int32_t) * (nt + 1), s);   // targets for the QR pass, and their count
        PCMS_CU(cudaMemsetAsync(qrl.as<int32_t>() + nt, 0, sizeof(int32_t), s));
        // fused apply: the FP64-assembled targets, whose rows k_rows64_apply applies
        DBuf l64(fused && mixed ? sizeof(int32_t) * (nt + 1) : 0, s);
        if (fused && mixed) PCMS_CU(cudaMemsetAsync(l64.as<int32_t>() + nt, 0, sizeof(int32_t), s));
        SolveArgs sa{};
        bases.apply(sa);
        sa.nt = nt;
        sa.counts = M.counts.as<int32_t>();
        sa.mom = mom.p;
        sa.lambda = P.lambda;
        if (deg >= 1) {
            sa.qr_list = qrl.as<int32_t>();
            sa.n_qr = qrl.as<int32_t>() + nt;
            sa.amp_qr = mixed ? AMP_QR_MIXED : AMP_QR_FP64;
        }
        if (fused && mixed) {
            sa.list64 = l64.as<int32_t>();
            sa.n64 = l64.as<int32_t>() + nt;
        }
        sa.y = y.as<double>();
        sa.yf = mixed ? yf.as<float2>() : nullptr;
        sa.flags = flags.as<int8_t>();
        sa.status = M.status.as<int8_t>();
        solve_tiers(dim, deg, MODE_MAP, mixed, plan, a, sa, nt, rc.as<float4>(), s);

        ShapeArgs sh{};
        sh.flags = flags.as<int8_t>();
        sh.rc = rc.as<float4>();
        sh.g = M.g;
        sh.ns = ns;
        sh.nt = nt;
        sh.sx64 = M.src.x64.as<double>();
        sh.hl0 = M.src.hl0.as<float4>();
        sh.hl1 = M.src.hl1.as<float2>();
        sh.tx64 = M.tgt.x64.as<double>();
        sh.thl0 = M.tgt.hl0.as<float4>();
        sh.thl1 = M.tgt.hl1.as<float2>();
        sh.lv = a.lv;
        sh.kexp = M.kexp.as<int32_t>();
        sh.offsets = M.offsets.as<int64_t>();
        sh.counts = M.counts.as<int32_t>();
        sh.cols = M.cols.as<int32_t>();
        sh.y = y.as<double>();
        sh.yf = mixed ? yf.as<float2>() : nullptr;
        sh.radius = P.radius;
        sh.weight = (int)P.weight;
        sh.vals = M.vals.p;
        if (fused) {
            // each row is applied to the fields as it is evaluated: no values stored, no SpMM
            const int fp = apply_fp_f32(fused->nf);
            DBuf fsd(sizeof(float) * fp * std::max<int64_t>(ns, 1), s);
            DBuf stage(sizeof(float) * fp * nt, s);
            fields_to_sorted_f32(M, fused->fields, fused->nf, fp, fsd.as<float>(), s);
            sh.fs = fsd.as<float>();
            sh.fp = fp;
            sh.status = M.status.as<int8_t>();
            sh.stage = stage.as<float>();
            shape_apply_any(dim, deg, G, sh, asm_blocks(nt, G), s);
            {
                PCMS_TRACE("mls_rows64_apply", s);
                rows64_apply_any(dim, deg, G, sh, l64.as<int32_t>(), l64.as<int32_t>() + nt, nt, s);
            }
            stage_to_caller_f32(M, stage.as<float>(), fp, fused->nf, fused->out, s);
        } else {
            shape_any(dim, deg, mixed, G, sh, asm_blocks(nt, G), s);
        }
        // the QR pass of the listed targets: an FP64 side table of their rows (rank failures
        // become ill-conditioned before the status counts below)
        if (deg >= 1) {
            int32_t hq = 0;
            PCMS_CU(cudaMemcpyAsync(&hq, qrl.as<int32_t>() + nt, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s));
            PCMS_CU(cudaStreamSynchronize(s));
            trace_count("mls_qr_rows", hq);
            qr_fix_map(M, qrl.as<int32_t>(), hq, s);
            if (fused) PCMS_CU(qr_apply(M, fused->fields, fused->nf, fused->out, s));
        }
        M.tgt.hl0.release();   // the targets' hi/lo coordinates only serve the assembly
        M.tgt.hl1.release();

        DBuf st(sizeof(unsigned long long) * 5, s);
        PCMS_CU(cudaMemsetAsync(st.p, 0, st.bytes, s));
        {
        PCMS_TRACE("mls_status_stats", s);
        k_stats<<<stats_blocks(nt), 256, 0, s>>>(M.status.as<int8_t>(), M.counts.as<int32_t>(),
                                                      M.kexp.as<int32_t>(), nt,
                                                      st.as<unsigned long long>());
        }
        PCMS_LAUNCH_CHECK("k_stats");
        unsigned long long hs[5];
        unsigned herr = 0;
        PCMS_CU(cudaMemcpyAsync(hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaMemcpyAsync(&herr, err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
        if (herr) fail(PCMS_ERR_CUDA, "internal: neighbour count above the row size");
        M.n_under = (int64_t)hs[0];
        M.n_ill = (int64_t)hs[1];
        M.max_count = (int64_t)hs[2];
        M.max_k = (int64_t)hs[3];
        M.nnz = (int64_t)hs[4];
        static const char* pair_names[2][3] = {
            {"mls_map_pairs_d2k0", "mls_map_pairs_d2k1", "mls_map_pairs_d2k2"},
            {"mls_map_pairs_d3k0", "mls_map_pairs_d3k1", "mls_map_pairs_d3k2"}};
        trace_count(pair_names[dim - 2][deg], M.nnz);   // the assembly's selected pairs
    }
}

// ------------------------------------------------------------------------------------
// radius search alone
// ------------------------------------------------------------------------------------
__global__ void k_counts_to_caller(int64_t nt, const int32_t* __restrict__ perm_t,
                                   const int32_t* __restrict__ c, const int32_t* __restrict__ k,
                                   int32_t* __restrict__ c_out, int32_t* __restrict__ k_out,
                                   int kadd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm_t[i];
        c_out[o] = c[i];
        if (k_out) k_out[o] = k[i] + kadd;
    }
}

void mls_count(const MlsParams& P0, const double* src, int64_t ns, const double* tgt, int64_t nt,
               const pcms_map_opts& o, int32_t* counts, int32_t* kexp, int64_t* total,
               cudaStream_t s) {
    if (P0.dim >= 4) return mls_nd_count(P0, src, ns, tgt, nt, counts, kexp, total, s);
    const MlsParams P = settle_growth(P0, src, ns, tgt, nt, o, s);
    const int dim = P.dim;
    const bool mixed = P.prec == PCMS_MIXED;
    BoxResult b = source_box(dim, src, ns, tgt, nt, o, s);
    const AsmPlan cplan = choose_plan(dim, 0, MODE_COUNT, ns, P.radius, b.lo, b.hi, mixed);
    Grid g = make_grid(dim, b.lo, b.hi, cplan.cell, MAX_CELLS, cplan.xs);
    SortedPoints S, Tp;
    sort_points(g, src, ns, true, mixed, S, s);
    sort_points(g, tgt, nt, false, mixed, Tp, s, true);
    const int G = cplan.G;
    DBuf c(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    DBuf k(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    DBuf off(sizeof(int64_t) * (nt + 1), s);
    if (nt > 0) {
        AsmArgs a = base_args(g, S, Tp, P);
        a.counts = c.as<int32_t>();
        a.kexp_out = k.as<int32_t>();
        assemble_any(dim, 0, mixed, MODE_COUNT, G, ACC_PLAIN, false, a, asm_blocks(nt, G), s);
        PCMS_TRACE("mls_counts_to_caller", s);
        k_counts_to_caller<<<thread_blocks(nt, 256), 256, 0, s>>>(
            nt, Tp.perm.as<int32_t>(), c.as<int32_t>(), k.as<int32_t>(), counts, kexp, P.kbase);
        PCMS_LAUNCH_CHECK("counts_to_caller");
    }
    if (total) {
        exclusive_scan<int64_t>(c.as<int32_t>(), off.as<int64_t>(), nt, s);
        PCMS_CU(cudaMemcpyAsync(total, off.as<int64_t>() + nt, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
    }
}

// ------------------------------------------------------------------------------------
// one-shot transfer (no operator)
// ------------------------------------------------------------------------------------
void mls_transfer(const MlsParams& P0, const double* src, int64_t ns, const double* tgt,
                  int64_t nt, const pcms_map_opts& o, const void* fields, int nf, void* out,
                  int8_t* status, cudaStream_t s, int64_t* n_under) {
    if (P0.dim >= 4)
        return mls_nd_transfer(P0, src, ns, tgt, nt, (const double*)fields, nf, (double*)out,
                               status, s, n_under);
    if (P0.prec == PCMS_MIXED && nf >= 3) {
        // several fields: one walk builds the operator's rows, which are applied to all the
        // fields as they are evaluated, instead of one fused walk per field
        MapImpl M;
        M.P = P0;
        M.ns = ns;
        M.nt = nt;
        M.stream = s;
        const FusedApply fa{(const float*)fields, nf, (float*)out};
        mls_create_map(M, src, tgt, o, &fa);
        if (status && nt > 0) mls_export(M, nullptr, nullptr, nullptr, status, nullptr, s);
        *n_under = M.n_under;
        return;
    }
    const MlsParams P = settle_growth(P0, src, ns, tgt, nt, o, s);
    const int dim = P.dim, deg = P.degree;
    const bool mixed = P.prec == PCMS_MIXED;
    *n_under = 0;
    BoxResult b = source_box(dim, src, ns, tgt, nt, o, s);
    const AsmPlan plan = choose_plan(dim, deg, MODE_FUSED, ns, P.radius, b.lo, b.hi, mixed);
    Grid g = make_grid(dim, b.lo, b.hi, plan.cell, MAX_CELLS, plan.xs);
    SortedPoints S, Tp;
    sort_points(g, src, ns, true, mixed, S, s);
    sort_points(g, tgt, nt, false, mixed, Tp, s, true);
    const int G = plan.G;
    const size_t fsz = mixed ? sizeof(float) : sizeof(double);
    DBuf fs(fsz * std::max<int64_t>(ns, 1), s);
    DBuf counts(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    DBuf kexp(sizeof(int32_t) * std::max<int64_t>(nt, 1), s);
    const int np = accp(dim, deg, MODE_FUSED);
    DBuf mom(mom_elem_bytes(mom_kind(mixed, plan.acc)) * np * std::max<int64_t>(nt, 1), s);
    BasisEstimate est;
    est.enable(mixed, plan, P, g, S, nt, s);
    DBuf qrl(sizeof(int32_t) * (nt + 1), s);   // targets for the QR pass, and their count
    PCMS_CU(cudaMemsetAsync(qrl.as<int32_t>() + nt, 0, sizeof(int32_t), s));
    for (int f = 0; f < nf; f++) {
        if (ns > 0) {
            PCMS_TRACE("mls_field_to_sorted", s);
            if (mixed)
                k_permute_field<float><<<thread_blocks(ns, 256), 256, 0, s>>>(
                    (const float*)fields + (int64_t)f * ns, S.inv.as<int32_t>(), ns, fs.as<float>());
            else
                k_permute_field<double><<<thread_blocks(ns, 256), 256, 0, s>>>(
                    (const double*)fields + (int64_t)f * ns, S.inv.as<int32_t>(), ns, fs.as<double>());
            PCMS_LAUNCH_CHECK("permute_field");
        }
        if (nt == 0) continue;
        AsmArgs a = base_args(g, S, Tp, P);
        a.counts = counts.as<int32_t>();
        a.kexp_out = kexp.as<int32_t>();
        a.field = fs.p;
        a.mom = mom.p;
        est.apply(a);
        assemble_any(dim, deg, mixed, MODE_FUSED, G, plan.acc, !mixed, a, asm_blocks(nt, G), s);
        SolveArgs sa{};
        est.apply(sa);
        sa.nt = nt;
        sa.counts = counts.as<int32_t>();
        sa.mom = mom.p;
        sa.lambda = P.lambda;
        sa.perm_t = Tp.perm.as<int32_t>();
        sa.out = (char*)out + fsz * (size_t)f * nt;
        sa.out_is_double = !mixed;
        sa.status = f == 0 ? status : nullptr;
        if (f == 0 && deg >= 1) {   // the same targets for every field: listed once
            sa.qr_list = qrl.as<int32_t>();
            sa.n_qr = qrl.as<int32_t>() + nt;
            sa.amp_qr = mixed ? AMP_QR_MIXED : AMP_QR_FP64;
        }
        solve_tiers(dim, deg, MODE_FUSED, mixed, plan, a, sa, nt, nullptr, s);
    }
    if (nt > 0 && deg >= 1)
        qr_fix_transfer(dim, deg, !mixed, g, S, Tp, kexp.as<int32_t>(), P.radius, (int)P.weight,
                        qrl.as<int32_t>(), qrl.as<int32_t>() + nt, fields, nf, out, status, s);
    if (status && P.min_neighbors == 0 && nt > 0) {
        DBuf st(sizeof(unsigned long long) * 4, s);
        PCMS_CU(cudaMemsetAsync(st.p, 0, st.bytes, s));
        // status is in caller order; counts/kexp only feed the max statistics here
        PCMS_TRACE("mls_status_stats", s);
        k_stats<<<stats_blocks(nt), 256, 0, s>>>(status, counts.as<int32_t>(),
                                                      kexp.as<int32_t>(), nt,
                                                      st.as<unsigned long long>());
        PCMS_LAUNCH_CHECK("k_stats");
        unsigned long long hs[4];
        PCMS_CU(cudaMemcpyAsync(hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaStreamSynchronize(s));
        *n_under = (int64_t)hs[0];
    }
}

}  // namespace pcms
