// pcms_internal.cuh -- shared declarations of the GB300 field-transfer library.
//
// Nothing here is visible through the C ABI (include/pcms.h). Internal errors are C++
// exceptions (PcmsError) that capi.cu converts into a pcms_status at the boundary.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>
#include <utility>

#include "pcms.h"

namespace pcms {

// ------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------
struct PcmsError {
    pcms_status status;
    std::string msg;
};

[[noreturn]] void fail(pcms_status st, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);

#define PCMS_CU(x) ::pcms::check_cuda((x), #x)
#define PCMS_LAUNCH_CHECK(name) ::pcms::check_cuda(cudaGetLastError(), name)

// ------------------------------------------------------------------------------------
// stream-ordered device memory (cudaMallocAsync / cudaFreeAsync on one stream)
// ------------------------------------------------------------------------------------
void ensure_mempool(int device);

// 1/x. On the device: Newton-Raphson from the FP32 reciprocal, two steps (2^-23 -> 2^-46 ->
// below FP64 rounding), about half the FP64 instructions of an IEEE division; IEEE division
// outside [1e-30, 1e30] and on the host.
__host__ __device__ __forceinline__ double recip64(double x) {
#ifdef __CUDA_ARCH__
    const double ax = fabs(x);
    if (ax > 1e-30 && ax < 1e30) {
        double r = (double)__frcp_rn((float)x);
        double e = fma(-x, r, 1.0);
        r = fma(r, e, r);
        e = fma(-x, r, 1.0);
        return fma(r, e, r);
    }
#endif
    return 1.0 / x;
}

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(size_t b, cudaStream_t st) { alloc(b, st); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; s = o.s;
            o.p = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t b, cudaStream_t st);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------------------------------
// uniform grid (Sec. 3.3 search structure)
// ------------------------------------------------------------------------------------
// Cells are h wide in y and z and h / xs wide in x (xs = 1, 2 or 4): finer x cells trim the
// x-rows of a ball's cells closer to its chords at the same number of rows. The x cells
// nest exactly in the h-wide columns: x / (h / xs) = xs * (x / h), a power-of-2 scaling.
struct Grid {
    int dim;
    int n[3];         // cells per axis (1 for unused axes); n[0] counts the h / xs cells
    int64_t ncell;
    double lo[3];     // origin (bounding-box minimum)
    double h, inv_h;  // cell edge (y, z) and its reciprocal
    int xs = 1;       // x cells per h

    __host__ __device__ double inv_hd(int d) const { return d == 0 ? inv_h * xs : inv_h; }
    __host__ __device__ int ncoarse_x() const { return (n[0] + xs - 1) / xs; }
};

// Cell edge h = r (1 + 2^-20) and cells per axis from a bounding box; h doubles until the
// grid has at most max_cells cells. Every point within r of a target lies in a cell at
// most 2^k cells away (per axis, in units of h) from the target's cell, for radius r 2^k.
Grid make_grid(int dim, const double* lo, const double* hi, double radius, int64_t max_cells,
               int xs = 1);
// The largest x subdivision in {4, 2, 1} whose grid (cell edge `cell`) has at most
// min(max_cells, 2 ns + 64) cells, so that the cell starts stay small next to the points.
int choose_xs(int dim, const double* lo, const double* hi, double cell, int64_t max_cells,
              int64_t ns);

// Where a point sits in the grid, in cell units: the cell coordinates (the floor, clamped
// to +-2^30, points outside the box included) and the FP32 position inside that cell. The
// radius-search walk starts from these. Unused axes give 0.
#ifdef __CUDACC__
__device__ __forceinline__ void point_cell(const Grid& g, int dim, const double* x, int4* cell,
                                           float4* frac) {
    int c[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f};
    for (int d = 0; d < dim; d++) {
        const double u = (x[d] - g.lo[d]) * g.inv_hd(d);
        double fl = floor(u);
        fl = fmin(fmax(fl, -1073741824.0), 1073741824.0);
        c[d] = (int)fl;
        f[d] = (float)(u - fl);
    }
    *cell = make_int4(c[0], c[1], c[2], 0);
    *frac = make_float4(f[0], f[1], f[2], 0.f);
}
#endif

// ------------------------------------------------------------------------------------
// points sorted by cell (counting sort)
// ------------------------------------------------------------------------------------
struct SortedPoints {
    int dim = 0;
    int64_t n = 0;
    DBuf cell_start;  // int32 [ncell+1]   (sources only)
    DBuf perm;        // int32 [n]: sorted position -> caller index
    DBuf inv;         // int32 [n]: caller index -> sorted position
    DBuf x64;         // float64 [dim][n] sorted coordinates
    DBuf hl0;         // float4 [n] (mixed path): 2D {xh,yh,xl,yl}; 3D {xh,yh,zh,xl}
    DBuf hl1;         // float2 [n] (mixed path, 3D): {yl,zl}
    DBuf cell;        // int4 [n] (targets): point_cell's cell coordinates
    DBuf frac;        // float4 [n] (targets): point_cell's position inside the cell
    DBuf xf;          // float32 [dim][n] (4D/5D sources): offsets from the grid origin
};

// Bounding boxes of pts (float64 [dim][n], dim <= 3) in one launch: per-block partial boxes (8 doubles per block, bbox_blocks(n)
// blocks) that the host combines after copying them back.
int bbox_blocks(int64_t n);
void launch_bbox_partials(int dim, const double* pts, int64_t n, double* part, cudaStream_t s);
void bbox_combine(const double* hpart, int64_t n, double* lo, double* hi, uint64_t* bad);
// Sort points by cell of grid g. with_start: also build cell_start (sources).
// with_hl: also write FP32 hi/lo coordinates relative to g.lo (mixed path).
void sort_points(const Grid& g, const double* pts, int64_t n, bool with_start, bool with_hl,
                 SortedPoints& out, cudaStream_t s, bool with_cell = false);

// Cell-sum pyramid of the sorted sources S (built with_start and with_hl). Level 0 holds per
// grid cell (sum of the sources' FP32 hi coordinates per axis, relative to g.lo; count);
// level j + 1 holds the sums over blocks of 2 x 2 (x 2) level-j entries, so an entry of level
// j covers 2^j cells per axis; level j has ceil(n_d / 2^j) entries along axis d, row-major,
// and starts at off[j]. pyramid_levels(g) levels, the last a single entry; pyramid_size
// gives the total entries (and fills off). Sums run in a fixed order (reproducible).
constexpr int PYR_MAX = 26;
int pyramid_levels(const Grid& g);
int64_t pyramid_size(const Grid& g, int levels, int64_t* off);
void cell_pyramid(const Grid& g, const SortedPoints& S, int levels, const int64_t* off,
                  float4* out, cudaStream_t s);

// Stable LSD radix sort (8-bit digits) of (key, value) pairs with keys < nkeys; k1/v1 are
// scratch of n entries. Returns the buffer (v0 or v1) holding the values in key order;
// keys_out, if given, receives the buffer holding the sorted keys.
uint32_t* radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n,
                           int64_t nkeys, cudaStream_t s, uint32_t** keys_out = nullptr);

// exclusive scan of int32 counts into out[0..n] (out[n] = total); T = int32_t or int64_t
template <typename T>
void exclusive_scan(const int32_t* in, T* out, int64_t n, cudaStream_t s);

// ------------------------------------------------------------------------------------
// compile-time monomial tables (graded-lex: by degree, then exponent of x descending,
// then exponent of y descending). 2D: 1, x, y, x^2, xy, y^2, ...; 3D: 1, x, y, z, x^2, xy,
// xz, y^2, yz, z^2, ...
// ------------------------------------------------------------------------------------
struct Exp3 {
    int e[3];
};

__host__ __device__ constexpr int binom(int n, int k) {
    int r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// monomials of degree <= deg in dim variables: C(dim + deg, deg)
__host__ __device__ constexpr int mono_count(int dim, int deg) {
    return deg < 0 ? 0 : binom(dim + deg, deg);
}

// Four and five variables (the FP64 path above 3D): the same graded-lex order, from a table
// of exponent vectors. Within a degree, vectors follow reverse-lexicographic order (e0
// descending, then e1, ...): from e, take the last i < dim-1 with e[i] > 0, lower e[i] by
// one, put the sum of e[i+1..] plus one into e[i+1] and clear the rest.
constexpr int ND_MAX_DIM = 5;
constexpr int ND_MAX_MOMENT_DEG = 4;   // moments of a quadratic basis
struct Exp5 {
    int e[ND_MAX_DIM];
};
template <int D>
struct MonoTab {
    static constexpr int N = binom(D + ND_MAX_MOMENT_DEG, ND_MAX_MOMENT_DEG);
    Exp5 x[N];
};
template <int D>
__host__ __device__ constexpr MonoTab<D> make_mono_tab() {
    MonoTab<D> t{};
    int idx = 0;
    for (int g = 0; g <= ND_MAX_MOMENT_DEG; ++g) {
        Exp5 e{};
        e.e[0] = g;
        for (;;) {
            t.x[idx++] = e;
            int i = -1;
            for (int j = 0; j < D - 1; ++j)
                if (e.e[j] > 0) i = j;
            if (i < 0) break;
            int rest = 0;
            for (int j = i + 1; j < D; ++j) rest += e.e[j];
            e.e[i] -= 1;
            e.e[i + 1] = rest + 1;
            for (int j = i + 2; j < D; ++j) e.e[j] = 0;
        }
    }
    return t;
}
template <int D>
__host__ __device__ constexpr Exp5 mono_exp_nd(int p) {
    return make_mono_tab<D>().x[p];
}
template <int D>
__host__ __device__ constexpr int mono_index_nd(const Exp5& e) {
    const MonoTab<D> t = make_mono_tab<D>();
    for (int p = 0; p < MonoTab<D>::N; ++p) {
        bool eq = true;
        for (int d = 0; d < D; ++d) eq = eq && t.x[p].e[d] == e.e[d];
        if (eq) return p;
    }
    return -1;
}
template <int D>
__host__ __device__ constexpr int mono_var_nd(int p) {
    const Exp5 x = mono_exp_nd<D>(p);
    for (int d = 0; d < D; ++d)
        if (x.e[d] > 0) return d;
    return 0;
}
template <int D>
__host__ __device__ constexpr int mono_parent_nd(int p) {
    Exp5 x = mono_exp_nd<D>(p);
    x.e[mono_var_nd<D>(p)] -= 1;
    return mono_index_nd<D>(x);
}
template <int D>
__host__ __device__ constexpr int mono_prod_nd(int k, int l) {
    const Exp5 a = mono_exp_nd<D>(k), b = mono_exp_nd<D>(l);
    Exp5 c{};
    for (int d = 0; d < D; ++d) c.e[d] = a.e[d] + b.e[d];
    return mono_index_nd<D>(c);
}

__host__ __device__ constexpr Exp3 mono_exp(int dim, int p) {
    int idx = 0;
    for (int g = 0; g <= 8; ++g)
        for (int e0 = g; e0 >= 0; --e0) {
            if (dim == 2) {
                if (idx == p) return Exp3{{e0, g - e0, 0}};
                ++idx;
            } else {
                for (int e1 = g - e0; e1 >= 0; --e1) {
                    if (idx == p) return Exp3{{e0, e1, g - e0 - e1}};
                    ++idx;
                }
            }
        }
    return Exp3{{-1, -1, -1}};
}

__host__ __device__ constexpr int mono_index(int dim, int e0, int e1, int e2) {
    for (int p = 0; p < mono_count(dim, 8); ++p) {
        Exp3 x = mono_exp(dim, p);
        if (x.e[0] == e0 && x.e[1] == e1 && x.e[2] == e2) return p;
    }
    return -1;
}

// first variable with a positive exponent, and the monomial with that exponent lowered
__host__ __device__ constexpr int mono_var(int dim, int p) {
    Exp3 x = mono_exp(dim, p);
    return x.e[0] > 0 ? 0 : (x.e[1] > 0 ? 1 : 2);
}

__host__ __device__ constexpr int mono_parent(int dim, int p) {
    Exp3 x = mono_exp(dim, p);
    int v = mono_var(dim, p);
    x.e[v] -= 1;
    return mono_index(dim, x.e[0], x.e[1], x.e[2]);
}

// index of the product of monomials k and l
__host__ __device__ constexpr int mono_prod(int dim, int k, int l) {
    if (dim == 4) return mono_prod_nd<4>(k, l);
    if (dim == 5) return mono_prod_nd<5>(k, l);
    Exp3 a = mono_exp(dim, k), b = mono_exp(dim, l);
    return mono_index(dim, a.e[0] + b.e[0], a.e[1] + b.e[1], a.e[2] + b.e[2]);
}

// static_for: calls f(std::integral_constant<int, I>) for I = 0 .. N-1 (indices are
// compile-time constants, so register arrays indexed by them stay in registers)
template <class F, int... Is>
__host__ __device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ constexpr int round_up4(int x) { return (x + 3) & ~3; }

// ------------------------------------------------------------------------------------
// MLS entry points (mls.cu)
// ------------------------------------------------------------------------------------
struct MlsParams {
    int dim, degree, m;
    pcms_precision prec;
    pcms_weight weight;
    double radius, lambda;
    int min_neighbors;
    int need;    // max(min_neighbors, m) if min_neighbors > 0 else 0
    int growth;  // pcms_growth
    int kbase;   // doublings already in radius (global growth), added to reported exponents
};

MlsParams make_mls_params(int dim, int degree, double radius, const pcms_map_opts& o);

// device bytes a request needs at most (sorted copies, operator, scratch), estimated from
// the sizes with the sources' bounding box taken as the unit box
int64_t estimate_mls_bytes(const MlsParams& P, int64_t ns, int64_t nt, int nf, bool keep_map);
int64_t estimate_mesh_bytes(int64_t nv, int64_t ntri, int64_t npts);

struct MapImpl {
    MlsParams P;
    Grid g;
    int64_t ns = 0, nt = 0, nnz = 0;
    cudaStream_t stream = nullptr;
    SortedPoints src, tgt;
    DBuf counts;     // int32 [nt] (sorted target order)
    DBuf kexp;       // int32 [nt]
    DBuf status;     // int8  [nt]
    DBuf offsets;    // int64 [nt+1] row starts; row t is [offsets[t], offsets[t] + counts[t])
    DBuf cols;       // int32 [nnz] sorted source positions
    DBuf vals;       // float64 or float32 [nnz]
    int64_t n_under = 0, n_ill = 0, max_count = 0, max_k = 0;
    // rows solved by Householder QR (qr_fix.cu): sorted targets, their (column, FP64 value)
    // pairs, QR_MAX per row, and the pairs used (-1: the assembled row stands)
    DBuf qr_list, qr_cols, qr_vals, qr_cnt;
    int qr_n = 0;
    int64_t device_bytes() const;
};

// fused: for a mixed map used once, evaluate its rows and apply them to these fields
// (float [nf][ns] -> out float [nf][nt]) in one pass instead of storing the values; the map
// then holds no values (M.vals empty) and is only fit to be destroyed
struct FusedApply {
    const float* fields;
    int nf;
    float* out;
};
void mls_create_map(MapImpl& M, const double* src, const double* tgt, const pcms_map_opts& o,
                    const FusedApply* fused = nullptr);
// apply pieces shared with the fused path (float fields): padded row width, fields into
// sorted order, staged rows back to caller order
int apply_fp_f32(int nf);
void fields_to_sorted_f32(const MapImpl& M, const float* fields, int nf, int fp, float* fs,
                          cudaStream_t s);
void stage_to_caller_f32(const MapImpl& M, const float* stage, int fp, int nf, float* out,
                         cudaStream_t s);
void mls_apply(MapImpl& M, const void* fields, int nf, void* out, cudaStream_t s);
// the same apply on the tensor cores (BF16 three-term splits, FP32 accumulation; apply_tc.cu)
void mls_apply_tc(MapImpl& M, const float* fields, int nf, float* out, cudaStream_t s);
// apply with caller-provided scratch of apply_scratch_bytes(M, nf) bytes (256-aligned base);
// allocates nothing, returns the first failing launch's status and names it in *where
int64_t apply_scratch_bytes(const MapImpl& M, int nf);
cudaError_t mls_apply_with_scratch(const MapImpl& M, const void* fields, int nf, void* out,
                                   void* scratch, cudaStream_t s, const char** where);
void mls_export(MapImpl& M, int64_t* offsets, int32_t* cols, double* vals, int8_t* status,
                int32_t* kexp, cudaStream_t s);
void mls_count(const MlsParams& P, const double* src, int64_t ns, const double* tgt, int64_t nt,
               const pcms_map_opts& o, int32_t* counts, int32_t* kexp, int64_t* total,
               cudaStream_t s);
void mls_transfer(const MlsParams& P, const double* src, int64_t ns, const double* tgt,
                  int64_t nt, const pcms_map_opts& o, const void* fields, int nf, void* out,
                  int8_t* status, cudaStream_t s, int64_t* n_under);

// Householder-QR pass for targets whose FP64 normal equations are too ill-conditioned
// (qr_fix.cu). One-shot: the listed sorted targets' values (all nf fields, caller order) and
// statuses are replaced. Map: the listed rows go to the map's FP64 side table (a failed rank
// test marks the target ill-conditioned); qr_apply then overwrites those targets' outputs
// after an apply (NaN for ill-conditioned ones), qr_export their exported rows.
void qr_fix_transfer(int dim, int deg, bool fp64, const Grid& g, const SortedPoints& S,
                     const SortedPoints& Tp, const int32_t* kexp, double radius, int weight,
                     const int32_t* list, const int32_t* n_list, const void* fields, int nf,
                     void* out, int8_t* status, cudaStream_t s);
void qr_fix_map(MapImpl& M, const int32_t* list, int n, cudaStream_t s);
cudaError_t qr_apply(const MapImpl& M, const void* fields, int nf, void* out, cudaStream_t s);
void qr_export(const MapImpl& M, const int64_t* off_out, int32_t* cols_out, double* vals_out,
               cudaStream_t s);
// Bounds on amp / rho (the error of an FP64 normal-equation solve is about amp / rho 2^-53
// of the field) above which a final FP64 solve is redone by QR: a quarter of the mixed
// path's 2e-5, a quarter of the FP64 path's 1e-12.
constexpr float AMP_QR_MIXED = 4.5e10f;
constexpr float AMP_QR_FP64 = 2.2e3f;

// four and five dimensions, FP64 (mls_nd.cu); the MLS entry points above dispatch here
void mls_nd_create_map(MapImpl& M, const double* src, const double* tgt);
void mls_nd_transfer(const MlsParams& P, const double* src, int64_t ns, const double* tgt,
                     int64_t nt, const double* fields, int nf, double* out, int8_t* status,
                     cudaStream_t s, int64_t* n_under);
void mls_nd_count(const MlsParams& P, const double* src, int64_t ns, const double* tgt, int64_t nt,
                  int32_t* counts, int32_t* kexp, int64_t* total, cudaStream_t s);

// the thread-local message returned by pcms_last_error (capi.cu)
void set_last_error_message(const std::string& msg);

// ------------------------------------------------------------------------------------
// mesh (mesh.cu)
// ------------------------------------------------------------------------------------
struct MeshImpl {
    int64_t nv = 0, ntri = 0, npairs = 0;
    cudaStream_t stream = nullptr;
    Grid g;
    double bbox[4];    // lo_x, lo_y, hi_x, hi_y of all vertices
    DBuf xy;           // float64 [2][nv]
    DBuf tri;          // int32 [3][ntri]
    DBuf cell_start;   // int32 [ncell+1]
    DBuf items;        // int32 [npairs] triangle ids, ascending within a cell
    DBuf tsign;        // int8 [ntri] orientation sign of each triangle (0 = degenerate)
    DBuf vhl;          // float4 [nv] vertex (x_hi, y_hi, x_lo, y_lo) relative to `origin`
    double origin[2];  // lower corner of the vertex box: the FP32 filter's frame
    float delta = 0.f; // absolute error allowance of the FP32 differences (2^-44 x extent)
    int use32 = 0;     // FP32 orientation filter usable (extent within [1e-30, 1e18])
    // built on first use by an L2 projection onto this mesh (mesh_adjacency)
    DBuf adj_start;    // int32 [nv+1]
    DBuf adj;          // int32 [3 ntri] entries 3 k + corner, ascending within a vertex
    DBuf tri_w;        // float64 [ntri] |T| / 12
};

void mesh_create(MeshImpl& M, const double* xy, int64_t nv, const int32_t* tri, int64_t ntri);
void mesh_locate(const MeshImpl& M, const double* pts, int64_t n, const double* field,
                 int32_t* elem, int8_t* edim, double* vals, cudaStream_t s);
void mesh_centroids(const MeshImpl& M, double* out, cudaStream_t s);
double mesh_integrate(const MeshImpl& M, const double* field, cudaStream_t s);

// conservative L2 projection of a P1 field between two meshes (projection.cu)
struct ProjectionResult {
    unsigned long long pairs;   // intersecting (source, target) triangle pairs
    int iterations;             // conjugate-gradient iterations
    double rel_residual;        // ||b - M f|| / ||b|| at the end
    double supermesh_area;
};
void mesh_adjacency(MeshImpl& M, cudaStream_t s);   // vertex -> triangles, |T| / 12 (cached)
ProjectionResult l2_project(const MeshImpl& S, const double* fs, MeshImpl& T, double* ft,
                            double tol, int max_iter, cudaStream_t s);

// number of SMs of the current device (cached)
int num_sms();

// plan tuning table (tune.cu; filled through pcms_tune_set)
struct TuneEntry {
    int dim, degree, mixed, mode, bucket;   // mode: 1 operator, 2 one-shot, 3 apply (bucket = fields)
    int lanes;                              // lanes per target (8 or 32)
    double cell_div;                        // grid cell edge = radius / cell_div
    int apply_form;                         // apply: 0 CUDA cores (FP32), 1 tensor cores (BF16 x 3)
};
int tune_bucket(double mean);   // floor(log2(expected neighbours)), 0 below 1
bool tune_lookup(int dim, int degree, bool mixed, int mode, int bucket, TuneEntry* out);

}  // namespace pcms

// the opaque handle behind pcms_map
struct pcms_map_s {
    pcms::MapImpl impl;
};
