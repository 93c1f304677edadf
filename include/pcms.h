/*
 * pcms.h -- C ABI of the GB300 field-transfer library (libpcms.so).
 *
 * Implements the data-parallel hot path of the field-mapping method of "PCMS: Parallel
 * Coupler for Multimodel Simulations" (arXiv 2510.18838):
 *   - meshless moving-least-squares (local weighted polynomial fitting) transfer with
 *     compactly supported radial weights (Sec. 3.2.1, Eq. 1, Table 1), behind
 *     pcms_create_map / pcms_apply_map / pcms_mls_transfer;
 *   - mesh point localization with lowest-order topological classification and
 *     barycentric (parametric) interpolation (Sec. 3.3), behind pcms_mesh_create /
 *     pcms_locate_interp.
 *
 * Conventions shared by every entry point:
 *   - Point arrays are structure-of-arrays float64 [dim][n] (x for all points, then y,
 *     then z). Every pointer argument named *_pts, fields, out, elem_ids, ... is a DEVICE
 *     pointer on the current CUDA device unless stated otherwise. The caller owns every
 *     buffer it passes; the library never frees or retains them past the call (it copies
 *     what a map or mesh needs into memory it owns).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is enqueued
 *     asynchronously on it; a call returns once its launches are enqueued, except where a
 *     sync is documented (a device-to-host read of a size or a status count).
 *   - Temporary and owned device memory comes from cudaMallocAsync on `stream`.
 *   - No C++ exception crosses this boundary. Every call returns a pcms_status; on an
 *     error pcms_last_error() returns a thread-local message. Inputs are validated on the
 *     host before anything is enqueued (NULL pointers, sizes, dim, degree, radius, NaN
 *     arguments); invalid arguments return PCMS_ERR_INVALID_ARG and enqueue nothing.
 *   - There is no CPU fallback: every step runs in the library's CUDA kernels (sm_103a).
 */
#ifndef PCMS_H
#define PCMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PCMS_OK = 0,
    PCMS_ERR_INVALID_ARG = 1,
    /* Sec. 3.2.1: with a user-given radius (min_neighbors == 0) some target has fewer
     * neighbours than basis terms; the map is still returned for inspection. */
    PCMS_ERR_UNDERDETERMINED = 2,
    PCMS_ERR_ILL_CONDITIONED = 3,
    PCMS_ERR_OUT_OF_MEMORY = 4,
    PCMS_ERR_TIMEOUT = 5,
    PCMS_ERR_CUDA = 6,
    PCMS_ERR_CAPACITY = 7
} pcms_status;

/* Arithmetic of the MLS path.
 * PCMS_FP64:  distances, weights, moments, solve and operator in FP64.
 * PCMS_MIXED: distance filter, weights and moment assembly in FP32 (coordinates as
 *             FP32 hi/lo pairs), FP64 solve with a conditioning guard (targets that fail
 *             it are re-assembled in FP64), FP32 operator and apply. Neighbour selection
 *             is decided in FP64 in both modes, so neighbour lists are identical. */
typedef enum { PCMS_FP64 = 0, PCMS_MIXED = 1 } pcms_precision;

/* Radial weights phi(q), q = r / r_c (Table 1 with a = 2, plus Wendland C2). */
typedef enum {
    PCMS_WENDLAND_C2 = 0, /* (1-q)^4 (4q+1) */
    PCMS_GAUSSIAN = 1,    /* exp(-(2q)^2) */
    PCMS_C4 = 2,          /* (5q^5+30q^4+72q^3+82q^2+36q+6)(1-q)^6 */
    PCMS_CONST = 3,       /* 1 */
    PCMS_NOOP = 4,        /* 1 (identity weight; selection stays the radius) */
    PCMS_MQ = 5,          /* sqrt(1+(2q)^2) */
    PCMS_IMQ = 6,         /* 1/sqrt(1+(2q)^2) */
    PCMS_TPS = 7,         /* (2q)^2 ln(2q) */
    PCMS_CUBIC = 8        /* (2q)^3 */
} pcms_weight;

/* Readings of the Sec. 3.2.1 minimum-count rule (pcms_map_opts.growth, min_neighbors > 0). */
typedef enum { PCMS_GROWTH_PER_TARGET = 0, PCMS_GROWTH_GLOBAL = 1 } pcms_growth;

/* per-target status codes (int8) */
enum { PCMS_TARGET_OK = 0, PCMS_TARGET_UNDERDETERMINED = 1, PCMS_TARGET_ILL_CONDITIONED = 2 };

typedef struct {
    pcms_precision precision; /* default PCMS_FP64 */
    pcms_weight weight;       /* default PCMS_WENDLAND_C2 */
    double lambda;            /* Tikhonov parameter of Eq. 1 (scaled basis), >= 0; default 0 */
    /* Sec. 3.2.1 selection modes. 0 (default): the radius is used as given and targets with
     * fewer than m neighbours are UNDERDETERMINED (value NaN). > 0: per target, the radius
     * is doubled until at least max(min_neighbors, m) sources are selected. */
    int min_neighbors;
    /* Optional: 1 if lo/hi bound every source point; saves one device-to-host read. */
    int domain_known;
    double lo[3], hi[3];
    /* How the radius grows when min_neighbors > 0. PCMS_GROWTH_PER_TARGET (default): each
     * target doubles its own radius. PCMS_GROWTH_GLOBAL: one radius, radius * 2^K, for every
     * target, with K the fewest doublings after which no target is short (K is also the
     * largest per-target doubling count, as counts only grow with the radius). The
     * reported radius doublings are then K for every target. */
    int growth;
} pcms_map_opts;

typedef struct pcms_map_s* pcms_map;
typedef struct pcms_mesh_s* pcms_mesh;

typedef struct {
    int dim, basis_degree, n_terms;
    pcms_precision precision;
    int64_t n_src, n_tgt, nnz;
    int64_t n_underdetermined, n_ill_conditioned; /* per-target status counts */
    int64_t max_neighbors, max_radius_doublings;
    int64_t device_bytes; /* memory owned by the map */
} pcms_map_info_t;

/* Library version (major*10000 + minor*100 + patch). */
int pcms_version(void);

/* Thread-local message describing the last error returned on this thread. */
const char* pcms_last_error(void);

/* Fill *opts with the defaults listed above. */
void pcms_map_opts_default(pcms_map_opts* opts);

/*
 * pcms_create_map -- build a cached MLS transfer operator (Sec. 3.2.1, Eq. 1).
 *   For every target point t_i, selects the sources with |s_j - t_i| < r (decided in FP64
 *   exactly as ((dx*dx + dy*dy) + dz*dz) < r*r, plus phi > 0), fits the weighted polynomial
 *   of degree `basis_degree` (0, 1 or 2; graded-lex monomials of (s - t)/r) and stores the
 *   shape functions N_ij so that f(t_i) = sum_j N_ij f(s_j).
 *   dim: 2, 3, 4 or 5 (fields in up to five dimensions; above 3D only PCMS_FP64 and no
 *   domain_known; the squared distance is summed left to right over all dimensions).
 *   src_pts: device float64 [dim][n_src]; tgt_pts: device float64 [dim][n_tgt].
 *   radius > 0. opts may be NULL (defaults). The map copies what it needs; inputs may be
 *   freed after the call returns and the stream has run.
 *   Syncs `stream` once to size the operator (and once more for the bounding box unless
 *   opts->domain_known). Returns PCMS_ERR_UNDERDETERMINED (map still created) when
 *   min_neighbors == 0 and some target has fewer than m neighbours.
 */
pcms_status pcms_create_map(int dim, const double* src_pts, int64_t n_src,
                            const double* tgt_pts, int64_t n_tgt, int basis_degree,
                            double radius, const pcms_map_opts* opts, void* stream,
                            pcms_map* out);

/*
 * pcms_apply_map -- evaluate out[f][i] = sum_j N_ij fields[f][j] for n_fields fields.
 *   fields: device [n_fields][n_src] in the caller's source order; out: device
 *   [n_fields][n_tgt] in the caller's target order. dtype is float64 for PCMS_FP64 maps and
 *   float32 for PCMS_MIXED maps. 1 <= n_fields <= 16. Targets whose status is not OK get NaN.
 *   Uses scratch of n_fields*(n_src+n_tgt) elements from cudaMallocAsync on `stream`.
 */
pcms_status pcms_apply_map(pcms_map map, const void* fields, int n_fields, void* out,
                           void* stream);

/*
 * pcms_mls_transfer -- one-shot MLS transfer of n_fields fields without storing an
 *   operator (same selection, weights and fit as pcms_create_map). One or two fields: the
 *   per-target fit is evaluated directly as c_0 = e_1^T G^-1 g, one walk per field. Three or
 *   more fields, PCMS_MIXED, 2D/3D: one walk builds each target's operator row, which is
 *   applied to all fields as it is evaluated and not stored. FP64 with three or more fields,
 *   and 4D/5D: a transient operator is built and applied. Arguments as pcms_create_map plus fields
 *   (device [n_fields][n_src], float64 for PCMS_FP64, float32 for PCMS_MIXED), out (device
 *   [n_fields][n_tgt], same dtype) and target_status (device int8 [n_tgt], may be NULL).
 *   1 <= n_fields <= 16. Syncs once for the bounding box unless opts->domain_known.
 *   Returns PCMS_ERR_UNDERDETERMINED only when target_status is non-NULL, min_neighbors
 *   == 0 and some target is underdetermined (this reads a count back: one more sync).
 */
pcms_status pcms_mls_transfer(int dim, const double* src_pts, int64_t n_src,
                              const double* tgt_pts, int64_t n_tgt, int basis_degree,
                              double radius, const pcms_map_opts* opts, const void* fields,
                              int n_fields, void* out, int8_t* target_status, void* stream);

/*
 * pcms_count_neighbors -- the radius search alone (Sec. 3.2.1 selection function, with the
 *   same minimum-count radius growth and the same FP64 decision as pcms_create_map).
 *   counts: device int32 [n_tgt] (caller target order), number of selected sources;
 *   radius_doublings: device int32 [n_tgt] or NULL; total: host int64 or NULL, the sum of
 *   counts (reading it syncs `stream`). Other arguments as pcms_create_map (the precision
 *   only selects the FP32 or FP64 distance filter; the decision is the same).
 */
pcms_status pcms_count_neighbors(int dim, const double* src_pts, int64_t n_src,
                                 const double* tgt_pts, int64_t n_tgt, int basis_degree,
                                 double radius, const pcms_map_opts* opts, int32_t* counts,
                                 int32_t* radius_doublings, int64_t* total, void* stream);

/*
 * Batched one-shot MLS transfer of many small, independent problems (Sec. 3.2.1, Eq. 1:
 * one local weighted fit per target, independent across targets and across problems).
 *
 * Each item is one transfer with its own sources, targets, radius, basis and fields, in
 * the mixed precision of PCMS_MIXED with a user-given radius (min_neighbors = 0) and
 * lambda = 0. Every item's selection, weights and fit are those of pcms_mls_transfer;
 * what differs is the execution. The items are grouped by (dim, basis_degree, lanes per
 * target); per group, one kernel sorts each item's sources into its own uniform grid (one
 * thread block per item: bounding box, cell keys, counting sort, sorted FP64 and FP32
 * hi/lo copies, fields in sorted order), and one persistent kernel takes (item, tile of
 * targets) work units from a counter and runs, per target, the radius walk, the FP32
 * moment assembly, the solve and the operator row applied to all fields, with the FP64
 * assembly and solve in the same kernel for targets whose conditioning estimate rejects
 * the FP32 moments. Neighbour counts from 10 to a few hundred per target, uneven across
 * items, share the GPU through the work counter. Item results do not depend on the other
 * items of the batch (bitwise).
 *
 *   src_pts/tgt_pts: device float64 [dim][n]; fields: device float32 [n_fields][n_src];
 *   out: device float32 [n_fields][n_tgt], NaN where the target's status is not OK;
 *   target_status: device int8 [n_tgt] or NULL (PCMS_TARGET_* codes).
 *   Limits: dim 2 or 3; basis_degree 0..2; 1 <= n_fields <= 16; n_src, n_tgt <=
 *   PCMS_BATCH_MAX_POINTS; radius finite and > 0; weight a pcms_weight.
 *   result (host int32 [n_items], may be NULL): per item PCMS_OK, or
 *   PCMS_ERR_INVALID_ARG when a point coordinate is not finite (that item's outputs are
 *   then unspecified). The call returns PCMS_ERR_INVALID_ARG, enqueuing nothing, when an
 *   item breaks a limit; otherwise it enqueues its work on `stream` and, when result is
 *   non-NULL, syncs `stream` once to read the per-item flags. Device scratch (about
 *   100 bytes per point plus 4 bytes per field and point) comes from cudaMallocAsync on
 *   `stream`.
 */
#define PCMS_BATCH_MAX_POINTS 131072
#define PCMS_BATCH_MAX_ITEMS 256

typedef struct {
    int dim;
    int basis_degree;
    double radius;
    pcms_weight weight;
    const double* src_pts;
    int64_t n_src;
    const double* tgt_pts;
    int64_t n_tgt;
    const float* fields;
    int n_fields;
    float* out;
    int8_t* target_status;
} pcms_batch_item;

pcms_status pcms_mls_transfer_batch(const pcms_batch_item* items, int n_items,
                                    int32_t* result, void* stream);

/*
 * pcms_apply_map_noalloc -- the same result as pcms_apply_map, for callers that must not
 *   allocate device memory while they run (for example a solver's time-step loop that keeps
 *   a fixed device-memory footprint after set-up, or code sharing the GPU with an
 *   application whose allocator owns the free memory). The paper has no counterpart: this
 *   is a deployment variant of the apply.
 *   Scratch comes from one fixed 32 MiB device array built into the library (held by every
 *   GPU that loads the library until the process exits); this call performs no device
 *   allocation or free. The scratch needed is about (n_src + n_tgt) * P * elem bytes, P =
 *   n_fields rounded up to 1, 4, 8 or 16 (float32 maps) or 1, 2, 4, 8, 16 (float64), elem =
 *   4 or 8; a map/field count needing more returns PCMS_ERR_CAPACITY and enqueues nothing.
 *   The first call on a device performs a one-time set-up for that device (it looks up the
 *   array's device address, which may load the library's device code); make that first
 *   call before any stream capture. Every call shares the one array and every element a
 *   call reads is written earlier by the same call, so nothing carries over between calls;
 *   calls whose work can overlap on the GPU (different streams, or host threads) race on
 *   the array and must be ordered by the caller. If a CUDA error from earlier work is
 *   pending on the calling thread, the call launches nothing, returns PCMS_ERR_CUDA and
 *   leaves that error pending for its owner. Arguments as pcms_apply_map.
 */
pcms_status pcms_apply_map_noalloc(pcms_map map, const void* fields, int n_fields, void* out,
                                   void* stream);

/*
 * pcms_apply_map_bf16 -- the result of pcms_apply_map for a PCMS_MIXED map (Sec. 3.2.1,
 *   Eq. 1, out = N F for up to 16 fields), computed on the tensor cores. Each FP32 operator
 *   value and field value is split into three BF16 terms (x = x_h + x_m + x_l to 2^-24 |x|);
 *   the six term products of order <= 2 (the BF16 product and its residual correction) are
 *   accumulated in FP32, so the accuracy is that of the FP32 apply. The fields are split once
 *   into BF16 planes in source order; per tile of 16 targets the nonzeros' field rows are
 *   gathered into shared memory and multiplied against the block-diagonal operator tile
 *   (mma.sync m16n8k16). Rows solved by QR (the map's FP64 side table) are applied as in
 *   pcms_apply_map. fields: device float32 [n_fields][n_src]; out: device float32
 *   [n_fields][n_tgt]; 1 <= n_fields <= 16; maps of dimension 2 or 3. Scratch: 96 bytes per
 *   source and 64 per target from cudaMallocAsync on `stream`. Asynchronous.
 */
pcms_status pcms_apply_map_bf16(pcms_map map, const float* fields, int n_fields, float* out,
                                void* stream);

/*
 * Plan tuning (no counterpart in the paper; runtime). The kernels' launch plan is chosen by
 * rules from the expected neighbour count n (sources per box volume times the ball): lanes per
 * target (8, or 32 from 160 neighbours), the grid's cell edge (r/3 in 2D, r/6 in 2D from 1000
 * neighbours, r/2 in 3D), and the CUDA-core apply. A tuning table replaces these choices
 * where it has an entry: for a (dim, degree, precision, mode, bucket = floor(log2 n)) the
 * lanes (8 or 32) and the cell divisor d (cell edge = radius / d, 1 <= d <= 8) measured
 * fastest; for mode PCMS_TUNE_APPLY (bucket = the field count, 1..16) the apply form that
 * pcms_apply_map uses for mixed maps (0: CUDA cores, FP32; 1: tensor cores, as
 * pcms_apply_map_bf16). The precision rules are not tuned: blocked compensation still takes
 * 32 lanes from 1000 neighbours. Results change only by rounding between plans. The python
 * package's tune module measures the candidates on seeded problems and writes the table.
 * pcms_tune_set replaces the whole table (n = 0 clears it) and may be called while other
 * threads run requests (they see the old or the new table). Invalid entries:
 * PCMS_ERR_INVALID_ARG, the table unchanged.
 */
enum { PCMS_TUNE_MAP = 1, PCMS_TUNE_ONESHOT = 2, PCMS_TUNE_APPLY = 3 };
typedef struct {
    int dim, degree;
    pcms_precision precision;
    int mode, bucket;
    int lanes;
    double cell_div;
    int apply_form;
} pcms_tune_entry;
pcms_status pcms_tune_set(const pcms_tune_entry* entries, int n);
int pcms_tune_count(void);
pcms_status pcms_tune_get(int i, pcms_tune_entry* entry);

/* Sizes and status counts of a map. Syncs the map's stream. */
pcms_status pcms_map_info(pcms_map map, pcms_map_info_t* info);

/*
 * pcms_map_export -- copy the operator out in the caller's orders (for tests/inspection).
 *   offsets: device int64 [n_tgt+1]; cols: device int32 [nnz] (caller source indices);
 *   vals: device float64 [nnz] or NULL; status: device int8 [n_tgt] or NULL;
 *   radius_doublings: device int32 [n_tgt] or NULL. Within a row the order of (col, val)
 *   pairs is unspecified.
 */
pcms_status pcms_map_export(pcms_map map, int64_t* offsets, int32_t* cols, double* vals,
                            int8_t* status, int32_t* radius_doublings, void* stream);

/* Release a map; its memory is freed on `stream` (stream order). NULL is a no-op. */
void pcms_map_destroy(pcms_map map, void* stream);

/*
 * pcms_mesh_create -- cache a triangle mesh and its uniform-grid search structure
 *   (Sec. 3.3). xy: device float64 [2][n_vertices]; tri: device int32 [3][n_tri] vertex
 *   ids (either orientation; zero-area triangles never contain a point). Syncs once for
 *   the bounding box and once for the number of (cell, triangle) pairs.
 */
pcms_status pcms_mesh_create(const double* xy, int64_t n_vertices, const int32_t* tri,
                             int64_t n_tri, void* stream, pcms_mesh* out);

/*
 * pcms_locate_interp -- point localization + barycentric interpolation (Sec. 3.3).
 *   tgt_pts: device float64 [2][n_pts]. elem_ids: device int32 [n_pts]: the smallest id
 *   among triangles whose closure contains the point (exact orientation predicates), -1
 *   if none. entity_dim (device int8 [n_pts] or NULL): dimension of the lowest-order mesh
 *   entity the point lies on (0 vertex, 1 edge, 2 face), -1 outside. values (device
 *   float64 [n_pts] or NULL, requires nodal_field device float64 [n_vertices]):
 *   l0 f0 + l1 f1 + l2 f2 with l0 = A(p,v1,v2)/A(v0,v1,v2), l1 = A(v0,p,v2)/A(v0,v1,v2),
 *   l2 = 1 - l0 - l1; NaN outside. Asynchronous.
 */
pcms_status pcms_locate_interp(pcms_mesh mesh, const double* tgt_pts, int64_t n_pts,
                               const double* nodal_field, int32_t* elem_ids,
                               int8_t* entity_dim, double* values, void* stream);

/*
 * pcms_mesh_centroids -- triangle centroids ((v0 + v1) + v2) / 3, written to centroids
 *   (device float64 [2][n_tri]): the element-centred points of the vertex <-> centroid
 *   round trip that measures accuracy and conservation (Sec. 3.2.1, Eq. 2 and Eq. 3).
 *   Asynchronous.
 */
pcms_status pcms_mesh_centroids(pcms_mesh mesh, double* centroids, void* stream);

/*
 * pcms_mesh_integrate -- integral over the mesh of the piecewise-linear interpolant of a
 *   nodal field (the integral of Eq. 3): the sum over triangles of |area| (f0 + f1 + f2) / 3,
 *   area = ((x1-x0)(y2-y0) - (y1-y0)(x2-x0)) / 2, in FP64 without contraction. The sum runs
 *   in a fixed order (per-block partial sums, then one block), so it is reproducible.
 *   nodal_field: device float64 [n_vertices]; *integral: host double, written after the
 *   call synchronises `stream`.
 */
pcms_status pcms_mesh_integrate(pcms_mesh mesh, const double* nodal_field, double* integral,
                                void* stream);

/*
 * pcms_l2_project -- conservative L2 projection of a piecewise-linear field (Sec. 3.2.2):
 *   f_t solves M f_t = b, M_AB = integral of N_A N_B (the target's consistent P1 mass matrix),
 *   b_A = integral of N_A f_s over the supermesh of the two meshes (each overlapping pair of
 *   triangles clipped to its common polygon, integrated exactly for P1 x P1). The integral
 *   of f_t equals that of f_s over the region both meshes cover, up to the solve's residual.
 *   src_field: device float64 [source vertices]; tgt_field: device float64 [target
 *   vertices] (written). M f = b is solved by Jacobi-preconditioned conjugate gradients to
 *   ||b - M f|| <= tol ||b|| (tol > 0, e.g. 1e-14) or max_iter iterations. info (host, may
 *   be NULL) receives the pair count, iterations, final relative residual and the area of
 *   the supermesh. Syncs `stream`. The target mesh caches its vertex-to-triangle lists.
 */
typedef struct {
    int64_t intersecting_pairs;
    int iterations;
    double relative_residual;
    double supermesh_area;
} pcms_projection_info;
pcms_status pcms_l2_project(pcms_mesh src_mesh, const double* src_field, pcms_mesh tgt_mesh,
                            double* tgt_field, double tol, int max_iter,
                            pcms_projection_info* info, void* stream);

/* Release a mesh (memory freed on `stream`). NULL is a no-op. */
void pcms_mesh_destroy(pcms_mesh mesh, void* stream);

/*
 * Serving: a continuous-batching request loop (no counterpart in the paper, which couples
 * applications through files/streams; this is the single-GPU runtime around the hot path).
 *
 * A server owns n_slots worker threads, each with its own non-blocking CUDA stream. Requests
 * are queued in submission order; the head request is admitted as soon as a slot is idle
 * and its device-memory estimate fits under mem_cap_bytes together with everything already
 * admitted or cached (least recently used cached operators are evicted first). Admitted
 * requests run concurrently on their slots' streams, so their kernels overlap on the GPU.
 * A request whose estimate alone exceeds the cap fails with PCMS_ERR_CAPACITY.
 * All pointers in a request are owned by the caller and must stay valid until the request
 * has completed. They are device pointers, or with host_io = 1 host pointers: the server
 * then copies the inputs the request needs to device memory on the slot's stream, runs it,
 * and copies the outputs back before reporting completion, so a request's copies overlap
 * other slots' kernels. Host buffers should be page-locked (cudaHostAlloc or
 * cudaHostRegister); pageable memory works but its copies do not overlap. The staging
 * memory is part of the request's reservation.
 */
typedef enum { PCMS_REQ_MLS = 0, PCMS_REQ_MESH = 1 } pcms_request_kind;

typedef struct {
    pcms_request_kind kind;
    /* MLS: dim, basis_degree, radius, opts, src_pts [dim][n_src], tgt_pts [dim][n_tgt],
     * fields [n_fields][n_src] (float32 for PCMS_MIXED, float64 for PCMS_FP64),
     * out [n_fields][n_tgt] (same dtype).
     * map_key >= 0: keep the operator cached under this key; a later request with the same
     * key and reuse_map = 1 applies the cached operator to its own fields. A reuse request
     * still passes the same geometry (src/tgt): it is used to rebuild the operator if it was
     * evicted, or if the request's scratch does not fit under the cap beside it (the
     * operator a request is admitted to apply is pinned before anything is evicted for it).
     * The cached operator must have the request's n_src, n_tgt, dim and precision, else the
     * request fails with PCMS_ERR_INVALID_ARG. map_key < 0: nothing is cached. */
    int dim, basis_degree;
    double radius;
    pcms_map_opts opts;
    const double* src_pts;
    int64_t n_src;
    const double* tgt_pts;
    int64_t n_tgt;
    const void* fields;
    int n_fields;
    void* out;
    int64_t map_key;
    int reuse_map;
    /* MESH: xy [2][n_vertices] (src_pts), n_vertices (n_src), tri [3][n_tri], points
     * (tgt_pts, n_tgt), nodal field (fields, float64 [n_vertices]), values out (out, float64
     * [n_tgt]), elem_ids (int32 [n_tgt], required). */
    const int32_t* tri;
    int64_t n_tri;
    int32_t* elem_ids;
    /* device bytes to reserve; 0 = estimate from the sizes */
    int64_t bytes_hint;
    /* 1: all buffers above are host memory, staged through the device by the server */
    int host_io;
} pcms_request;

typedef struct {
    int64_t ticket;
    pcms_status status;
    double t_submit, t_start, t_end; /* seconds on the server's monotonic clock */
    int64_t bytes_reserved;
    int used_cached_map;
} pcms_request_result;

typedef struct pcms_server_s* pcms_server;

/* Start a server on the current device. n_slots in 1..64, mem_cap_bytes > 0. */
pcms_status pcms_server_create(int n_slots, int64_t mem_cap_bytes, pcms_server* out);
/* Queue a request (copied); *ticket receives its id (0, 1, 2, ...). Never blocks on the GPU. */
pcms_status pcms_server_submit(pcms_server s, const pcms_request* req, int64_t* ticket);
/* Up to max_results completed requests not yet returned, in completion order. Waits up to
 * timeout_s for at least one (0 = do not wait). *n_results may be 0 (PCMS_OK). */
pcms_status pcms_server_poll(pcms_server s, pcms_request_result* results, int max_results,
                             double timeout_s, int* n_results);
/* Wait until every submitted request has completed; PCMS_ERR_TIMEOUT after timeout_s. */
pcms_status pcms_server_drain(pcms_server s, double timeout_s);
/* Current time on the server's monotonic clock (seconds). */
double pcms_server_now(pcms_server s);
/* Batching of small requests (no counterpart in the paper; runtime). A request that is a
 * one-shot PCMS_MIXED MLS transfer (map_key < 0, reuse_map = 0) with min_neighbors = 0,
 * lambda = 0 and at most max_points sources and targets goes through the batched path of
 * pcms_mls_transfer_batch: when a slot takes such a request from the head of the queue, it
 * also takes the other queued requests of that kind that fit under the cap (up to
 * PCMS_BATCH_MAX_ITEMS requests and 2^21 targets, in queue order) and runs them together,
 * one CUDA graph replay per shape class. Results are those of pcms_mls_transfer_batch and do
 * not depend on which requests share a batch. max_points = 0 turns batching off; values
 * above PCMS_BATCH_MAX_POINTS are clamped. Default 8192. Takes effect for requests
 * admitted after the call. */
pcms_status pcms_server_set_batching(pcms_server s, int64_t max_points);
/* Batches run so far and the requests they held. */
pcms_status pcms_server_batch_stats(pcms_server s, int64_t* n_batches, int64_t* n_batched);
/* Bytes currently reserved by admitted requests plus cached operators, and the peak. */
pcms_status pcms_server_memory(pcms_server s, int64_t* in_use, int64_t* peak,
                               int64_t* cached_maps);
/* Drain, stop the workers, free cached operators. NULL is a no-op. */
void pcms_server_destroy(pcms_server s);

/*
 * Kernel tracing (no counterpart in the paper; instrumentation). mode 1 (timing): every
 * library kernel launch is bracketed by a CUDA event pair recorded on the stream it is
 * launched on, elapsed times are accumulated per kernel name, and work counts are recorded
 * as "count:<name>" entries (some of which cost a small extra kernel and a sync: pairs per
 * precision tier). mode 2 (count): launches are only counted per kernel name (total_ms 0),
 * with no events and no extra work. Any other non-zero mode is mode 1. A non-zero mode
 * clears the table; 0 stops recording and keeps it. pcms_trace_count and pcms_trace_get
 * synchronise on the recorded events. Thread-safe. Off by default.
 */
pcms_status pcms_trace_enable(int mode);
int pcms_trace_count(void);
/* Entry `index` (0 <= index < pcms_trace_count()): name (NUL-terminated, truncated to
 * name_len), number of launches and total milliseconds. PCMS_ERR_INVALID_ARG if out of range. */
pcms_status pcms_trace_get(int index, char* name, int name_len, int64_t* launches,
                           double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* PCMS_H */
