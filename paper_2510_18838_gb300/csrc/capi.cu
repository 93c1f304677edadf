// capi.cu -- the extern "C" boundary declared in include/pcms.h: argument validation,
// handle lifetime, and conversion of internal errors into pcms_status codes. No C++
// exception crosses this file's functions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "pcms_batch.cuh"
#include "pcms_internal.cuh"
#include "trace.cuh"

struct pcms_mesh_s {
    pcms::MeshImpl impl;
};

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace pcms {
void set_last_error_message(const std::string& msg) { g_last_error = msg; }
}  // namespace pcms

namespace {

pcms_status set_error(pcms_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

template <class F>
pcms_status guarded(const char* fn, F&& f) {
    try {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return set_error(PCMS_ERR_CUDA, std::string(fn) + ": no CUDA device");
        }
        pcms::ensure_mempool(dev);
        pcms_status st = f();
        if (st == PCMS_OK) g_last_error.clear();
        return st;
    } catch (const pcms::PcmsError& e) {
        return set_error(e.status, std::string(fn) + ": " + e.msg);
    } catch (const std::bad_alloc&) {
        return set_error(PCMS_ERR_OUT_OF_MEMORY, std::string(fn) + ": host allocation failed");
    } catch (...) {
        return set_error(PCMS_ERR_CUDA, std::string(fn) + ": unexpected internal error");
    }
}

#define REQUIRE(cond, msg)                                        \
    do {                                                          \
        if (!(cond)) return set_error(PCMS_ERR_INVALID_ARG, msg); \
    } while (0)

int num_terms(int dim, int degree) {
    if (degree == 0) return 1;
    if (degree == 1) return dim + 1;
    return dim == 2 ? 6 : 10;
}

pcms_status check_mls_args(const char* fn, int dim, const double* src, int64_t ns,
                           const double* tgt, int64_t nt, int degree, double radius,
                           const pcms_map_opts& o) {
    std::string f(fn);
    REQUIRE(dim >= 2 && dim <= 5, f + ": dim must be 2, 3, 4 or 5");
    REQUIRE(dim <= 3 || o.precision == PCMS_FP64,
            f + ": above 3D only the FP64 path exists (precision must be PCMS_FP64)");
    REQUIRE(dim <= 3 || !o.domain_known, f + ": domain_known covers at most 3 dimensions");
    REQUIRE(degree >= 0 && degree <= 2, f + ": basis_degree must be 0, 1 or 2");
    REQUIRE(std::isfinite(radius) && radius > 0.0, f + ": radius must be finite and > 0");
    REQUIRE(ns >= 0 && nt >= 0, f + ": negative point count");
    REQUIRE(ns < (int64_t(1) << 31) - 1 && nt < (int64_t(1) << 31) - 1,
            f + ": point counts must be below 2^31");
    REQUIRE(ns == 0 || src != nullptr, f + ": src_pts is NULL");
    REQUIRE(nt == 0 || tgt != nullptr, f + ": tgt_pts is NULL");
    REQUIRE(o.precision == PCMS_FP64 || o.precision == PCMS_MIXED, f + ": bad precision");
    REQUIRE((int)o.weight >= 0 && (int)o.weight <= 8, f + ": bad weight kind");
    REQUIRE(std::isfinite(o.lambda) && o.lambda >= 0.0, f + ": lambda must be finite and >= 0");
    REQUIRE(o.min_neighbors >= 0, f + ": min_neighbors must be >= 0");
    REQUIRE(o.growth == PCMS_GROWTH_PER_TARGET || o.growth == PCMS_GROWTH_GLOBAL,
            f + ": growth must be PCMS_GROWTH_PER_TARGET or PCMS_GROWTH_GLOBAL");
    if (o.domain_known) {
        for (int d = 0; d < dim; d++)
            REQUIRE(std::isfinite(o.lo[d]) && std::isfinite(o.hi[d]) && o.lo[d] <= o.hi[d],
                    f + ": bad domain box");
    }
    return PCMS_OK;
}

pcms::MlsParams make_params(int dim, int degree, double radius, const pcms_map_opts& o) {
    return pcms::make_mls_params(dim, degree, radius, o);
}

}  // namespace

extern "C" {

int pcms_version(void) { return 10000; }

const char* pcms_last_error(void) { return g_last_error.c_str(); }

void pcms_map_opts_default(pcms_map_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = PCMS_FP64;
    o->weight = PCMS_WENDLAND_C2;
    o->lambda = 0.0;
    o->min_neighbors = 0;
    o->domain_known = 0;
    o->growth = PCMS_GROWTH_PER_TARGET;
}

pcms_status pcms_create_map(int dim, const double* src_pts, int64_t n_src, const double* tgt_pts,
                            int64_t n_tgt, int basis_degree, double radius,
                            const pcms_map_opts* opts, void* stream, pcms_map* out) {
    if (!out) return set_error(PCMS_ERR_INVALID_ARG, "pcms_create_map: out is NULL");
    *out = nullptr;
    pcms_map_opts o;
    pcms_map_opts_default(&o);
    if (opts) o = *opts;
    pcms_status st = check_mls_args("pcms_create_map", dim, src_pts, n_src, tgt_pts, n_tgt,
                                    basis_degree, radius, o);
    if (st != PCMS_OK) return st;
    return guarded("pcms_create_map", [&]() -> pcms_status {
        pcms_map_s* m = new pcms_map_s();
        m->impl.P = make_params(dim, basis_degree, radius, o);
        m->impl.ns = n_src;
        m->impl.nt = n_tgt;
        m->impl.stream = (cudaStream_t)stream;
        try {
            pcms::mls_create_map(m->impl, src_pts, tgt_pts, o);
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
        if (o.min_neighbors == 0 && m->impl.n_under > 0)
            return set_error(PCMS_ERR_UNDERDETERMINED,
                             "pcms_create_map: " + std::to_string(m->impl.n_under) +
                                 " target(s) have fewer neighbours than basis terms");
        return PCMS_OK;
    });
}

pcms_status pcms_apply_map(pcms_map map, const void* fields, int n_fields, void* out,
                           void* stream) {
    REQUIRE(map != nullptr, "pcms_apply_map: map is NULL");
    REQUIRE(n_fields >= 1 && n_fields <= 16, "pcms_apply_map: n_fields must be in 1..16");
    REQUIRE(map->impl.ns == 0 || fields != nullptr, "pcms_apply_map: fields is NULL");
    REQUIRE(map->impl.nt == 0 || out != nullptr, "pcms_apply_map: out is NULL");
    return guarded("pcms_apply_map", [&]() -> pcms_status {
        pcms::mls_apply(map->impl, fields, n_fields, out, (cudaStream_t)stream);
        return PCMS_OK;
    });
}

pcms_status pcms_apply_map_bf16(pcms_map map, const float* fields, int n_fields, float* out,
                                void* stream) {
    REQUIRE(map != nullptr, "pcms_apply_map_bf16: map is NULL");
    REQUIRE(map->impl.P.prec == PCMS_MIXED, "pcms_apply_map_bf16: the map must be PCMS_MIXED");
    REQUIRE(map->impl.P.dim <= 3, "pcms_apply_map_bf16: maps of dimension 2 or 3");
    REQUIRE(n_fields >= 1 && n_fields <= 16, "pcms_apply_map_bf16: n_fields must be in 1..16");
    REQUIRE(map->impl.ns == 0 || fields != nullptr, "pcms_apply_map_bf16: fields is NULL");
    REQUIRE(map->impl.nt == 0 || out != nullptr, "pcms_apply_map_bf16: out is NULL");
    return guarded("pcms_apply_map_bf16", [&]() -> pcms_status {
        pcms::mls_apply_tc(map->impl, fields, n_fields, out, (cudaStream_t)stream);
        return PCMS_OK;
    });
}

pcms_status pcms_mls_transfer_batch(const pcms_batch_item* items, int n_items,
                                    int32_t* result, void* stream) {
    REQUIRE(n_items >= 0 && n_items <= PCMS_BATCH_MAX_ITEMS,
            "pcms_mls_transfer_batch: n_items must be in 0..PCMS_BATCH_MAX_ITEMS");
    REQUIRE(n_items == 0 || items != nullptr, "pcms_mls_transfer_batch: items is NULL");
    for (int i = 0; i < n_items; i++) {
        const std::string e = pcms::batch_check_item(items[i]);
        if (!e.empty())
            return set_error(PCMS_ERR_INVALID_ARG, "pcms_mls_transfer_batch: item " +
                                                       std::to_string(i) + ": " + e);
    }
    return guarded("pcms_mls_transfer_batch", [&]() -> pcms_status {
        // one executor per host thread and device (direct launches, table copied from
        // pageable memory, so consecutive calls never wait on each other's table)
        thread_local std::unique_ptr<pcms::BatchExec> ex[64];
        int dev = 0;
        PCMS_CU(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) pcms::fail(PCMS_ERR_CUDA, "device ordinal above 63");
        if (!ex[dev]) ex[dev].reset(new pcms::BatchExec(false));
        ex[dev]->run(items, n_items, result, (cudaStream_t)stream);
        return PCMS_OK;
    });
}

pcms_status pcms_mls_transfer(int dim, const double* src_pts, int64_t n_src,
                              const double* tgt_pts, int64_t n_tgt, int basis_degree,
                              double radius, const pcms_map_opts* opts, const void* fields,
                              int n_fields, void* out, int8_t* target_status, void* stream) {
    pcms_map_opts o;
    pcms_map_opts_default(&o);
    if (opts) o = *opts;
    pcms_status st = check_mls_args("pcms_mls_transfer", dim, src_pts, n_src, tgt_pts, n_tgt,
                                    basis_degree, radius, o);
    if (st != PCMS_OK) return st;
    REQUIRE(n_fields >= 1 && n_fields <= 16, "pcms_mls_transfer: n_fields must be in 1..16");
    REQUIRE(n_src == 0 || fields != nullptr, "pcms_mls_transfer: fields is NULL");
    REQUIRE(n_tgt == 0 || out != nullptr, "pcms_mls_transfer: out is NULL");
    return guarded("pcms_mls_transfer", [&]() -> pcms_status {
        cudaStream_t s = (cudaStream_t)stream;
        pcms::MlsParams P = make_params(dim, basis_degree, radius, o);
        int64_t n_under = 0;
        if (n_fields <= 2 || (o.precision == PCMS_MIXED && dim <= 3)) {
            // one or two fields: fused walks; several mixed fields: the operator's rows
            // applied as they are evaluated, without storing them
            pcms::mls_transfer(P, src_pts, n_src, tgt_pts, n_tgt, o, fields, n_fields, out,
                               target_status, s, &n_under);
        } else {
            // several FP64 fields: build a transient operator once and apply it
            pcms::MapImpl M;
            M.P = P;
            M.ns = n_src;
            M.nt = n_tgt;
            M.stream = s;
            pcms::mls_create_map(M, src_pts, tgt_pts, o);
            pcms::mls_apply(M, fields, n_fields, out, s);
            if (target_status)
                pcms::mls_export(M, nullptr, nullptr, nullptr, target_status, nullptr, s);
            n_under = M.n_under;
        }
        if (target_status && o.min_neighbors == 0 && n_under > 0)
            return set_error(PCMS_ERR_UNDERDETERMINED,
                             "pcms_mls_transfer: " + std::to_string(n_under) +
                                 " target(s) have fewer neighbours than basis terms");
        return PCMS_OK;
    });
}

pcms_status pcms_count_neighbors(int dim, const double* src_pts, int64_t n_src,
                                 const double* tgt_pts, int64_t n_tgt, int basis_degree,
                                 double radius, const pcms_map_opts* opts, int32_t* counts,
                                 int32_t* radius_doublings, int64_t* total, void* stream) {
    pcms_map_opts o;
    pcms_map_opts_default(&o);
    if (opts) o = *opts;
    pcms_status st = check_mls_args("pcms_count_neighbors", dim, src_pts, n_src, tgt_pts, n_tgt,
                                    basis_degree, radius, o);
    if (st != PCMS_OK) return st;
    REQUIRE(n_tgt == 0 || counts != nullptr, "pcms_count_neighbors: counts is NULL");
    return guarded("pcms_count_neighbors", [&]() -> pcms_status {
        pcms::MlsParams P = make_params(dim, basis_degree, radius, o);
        pcms::mls_count(P, src_pts, n_src, tgt_pts, n_tgt, o, counts, radius_doublings, total,
                        (cudaStream_t)stream);
        return PCMS_OK;
    });
}

pcms_status pcms_map_info(pcms_map map, pcms_map_info_t* info) {
    REQUIRE(map != nullptr && info != nullptr, "pcms_map_info: NULL argument");
    return guarded("pcms_map_info", [&]() -> pcms_status {
        const pcms::MapImpl& M = map->impl;
        PCMS_CU(cudaStreamSynchronize(M.stream));
        info->dim = M.P.dim;
        info->basis_degree = M.P.degree;
        info->n_terms = M.P.m;
        info->precision = M.P.prec;
        info->n_src = M.ns;
        info->n_tgt = M.nt;
        info->nnz = M.nnz;
        info->n_underdetermined = M.n_under;
        info->n_ill_conditioned = M.n_ill;
        info->max_neighbors = M.max_count;
        info->max_radius_doublings = M.max_k + M.P.kbase;
        info->device_bytes = M.device_bytes();
        return PCMS_OK;
    });
}

pcms_status pcms_map_export(pcms_map map, int64_t* offsets, int32_t* cols, double* vals,
                            int8_t* status, int32_t* radius_doublings, void* stream) {
    REQUIRE(map != nullptr, "pcms_map_export: map is NULL");
    REQUIRE((offsets == nullptr) == (cols == nullptr),
            "pcms_map_export: offsets and cols go together");
    REQUIRE(vals == nullptr || cols != nullptr, "pcms_map_export: vals needs cols");
    return guarded("pcms_map_export", [&]() -> pcms_status {
        pcms::mls_export(map->impl, offsets, cols, vals, status, radius_doublings,
                         (cudaStream_t)stream);
        return PCMS_OK;
    });
}

void pcms_map_destroy(pcms_map map, void* stream) {
    if (!map) return;
    // re-home every buffer on the caller's stream so the frees are ordered after its work
    cudaStream_t s = (cudaStream_t)stream;
    pcms::MapImpl& M = map->impl;
    pcms::DBuf* bufs[] = {&M.src.cell_start, &M.src.perm, &M.src.inv, &M.src.x64, &M.src.hl0,
                          &M.src.hl1, &M.tgt.cell_start, &M.tgt.perm, &M.tgt.inv, &M.tgt.x64,
                          &M.tgt.hl0, &M.tgt.hl1, &M.counts, &M.kexp, &M.status, &M.offsets,
                          &M.cols, &M.vals};
    for (pcms::DBuf* b : bufs) {
        b->s = s;
        b->release();
    }
    delete map;
}

pcms_status pcms_mesh_create(const double* xy, int64_t n_vertices, const int32_t* tri,
                             int64_t n_tri, void* stream, pcms_mesh* out) {
    if (!out) return set_error(PCMS_ERR_INVALID_ARG, "pcms_mesh_create: out is NULL");
    *out = nullptr;
    REQUIRE(n_vertices >= 0 && n_tri >= 0, "pcms_mesh_create: negative size");
    REQUIRE(n_vertices < (int64_t(1) << 31) - 1 && n_tri < (int64_t(1) << 30),
            "pcms_mesh_create: mesh too large");
    REQUIRE(n_vertices == 0 || xy != nullptr, "pcms_mesh_create: xy is NULL");
    REQUIRE(n_tri == 0 || tri != nullptr, "pcms_mesh_create: tri is NULL");
    return guarded("pcms_mesh_create", [&]() -> pcms_status {
        pcms_mesh_s* m = new pcms_mesh_s();
        m->impl.stream = (cudaStream_t)stream;
        try {
            pcms::mesh_create(m->impl, xy, n_vertices, tri, n_tri);
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
        return PCMS_OK;
    });
}

pcms_status pcms_locate_interp(pcms_mesh mesh, const double* tgt_pts, int64_t n_pts,
                               const double* nodal_field, int32_t* elem_ids, int8_t* entity_dim,
                               double* values, void* stream) {
    REQUIRE(mesh != nullptr, "pcms_locate_interp: mesh is NULL");
    REQUIRE(n_pts >= 0, "pcms_locate_interp: negative n_pts");
    REQUIRE(n_pts == 0 || (tgt_pts != nullptr && elem_ids != nullptr),
            "pcms_locate_interp: NULL tgt_pts or elem_ids");
    REQUIRE(values == nullptr || nodal_field != nullptr,
            "pcms_locate_interp: values requires nodal_field");
    return guarded("pcms_locate_interp", [&]() -> pcms_status {
        pcms::mesh_locate(mesh->impl, tgt_pts, n_pts, values ? nodal_field : nullptr, elem_ids,
                          entity_dim, values, (cudaStream_t)stream);
        return PCMS_OK;
    });
}

pcms_status pcms_mesh_centroids(pcms_mesh mesh, double* centroids, void* stream) {
    REQUIRE(mesh != nullptr, "pcms_mesh_centroids: mesh is NULL");
    REQUIRE(mesh->impl.ntri == 0 || centroids != nullptr, "pcms_mesh_centroids: centroids is NULL");
    return guarded("pcms_mesh_centroids", [&]() -> pcms_status {
        pcms::mesh_centroids(mesh->impl, centroids, (cudaStream_t)stream);
        return PCMS_OK;
    });
}

pcms_status pcms_mesh_integrate(pcms_mesh mesh, const double* nodal_field, double* integral,
                                void* stream) {
    REQUIRE(mesh != nullptr && integral != nullptr, "pcms_mesh_integrate: NULL argument");
    REQUIRE(mesh->impl.nv == 0 || nodal_field != nullptr, "pcms_mesh_integrate: nodal_field is NULL");
    return guarded("pcms_mesh_integrate", [&]() -> pcms_status {
        *integral = pcms::mesh_integrate(mesh->impl, nodal_field, (cudaStream_t)stream);
        return PCMS_OK;
    });
}

pcms_status pcms_l2_project(pcms_mesh src_mesh, const double* src_field, pcms_mesh tgt_mesh,
                            double* tgt_field, double tol, int max_iter,
                            pcms_projection_info* info, void* stream) {
    REQUIRE(src_mesh != nullptr && tgt_mesh != nullptr, "pcms_l2_project: mesh is NULL");
    REQUIRE(src_mesh->impl.nv == 0 || src_field != nullptr, "pcms_l2_project: src_field is NULL");
    REQUIRE(tgt_mesh->impl.nv == 0 || tgt_field != nullptr, "pcms_l2_project: tgt_field is NULL");
    REQUIRE(std::isfinite(tol) && tol > 0.0, "pcms_l2_project: tol must be finite and > 0");
    REQUIRE(max_iter >= 1, "pcms_l2_project: max_iter must be >= 1");
    return guarded("pcms_l2_project", [&]() -> pcms_status {
        const pcms::ProjectionResult r = pcms::l2_project(src_mesh->impl, src_field, tgt_mesh->impl,
                                                          tgt_field, tol, max_iter,
                                                          (cudaStream_t)stream);
        if (info) {
            info->intersecting_pairs = (int64_t)r.pairs;
            info->iterations = r.iterations;
            info->relative_residual = r.rel_residual;
            info->supermesh_area = r.supermesh_area;
        }
        return PCMS_OK;
    });
}

pcms_status pcms_trace_enable(int mode) {
    pcms::trace_enable(mode);
    return PCMS_OK;
}

int pcms_trace_count(void) { return pcms::trace_count(); }

pcms_status pcms_trace_get(int index, char* name, int name_len, int64_t* launches,
                           double* total_ms) {
    if (!pcms::trace_get(index, name, name_len, launches, total_ms))
        return set_error(PCMS_ERR_INVALID_ARG, "pcms_trace_get: index out of range");
    return PCMS_OK;
}

void pcms_mesh_destroy(pcms_mesh mesh, void* stream) {
    if (!mesh) return;
    cudaStream_t s = (cudaStream_t)stream;
    pcms::MeshImpl& M = mesh->impl;
    pcms::DBuf* bufs[] = {&M.xy, &M.tri, &M.cell_start, &M.items, &M.tsign, &M.vhl,
                          &M.adj_start, &M.adj, &M.tri_w};
    for (pcms::DBuf* b : bufs) {
        b->s = s;
        b->release();
    }
    delete mesh;
}

}  // extern "C"
