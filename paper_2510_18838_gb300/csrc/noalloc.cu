// noalloc.cu -- pcms_apply_map_noalloc: the operator apply for callers that must not
// allocate device memory while they run.
//
// Some callers cannot allocate at the point where they apply a transfer operator: a
// coupled solver's time-step loop that has to keep a fixed device-memory footprint after
// its set-up phase, code that shares the GPU with an application whose allocator already
// owns the free memory, or latency-critical paths where an allocation may synchronise the
// device or fail under memory pressure. pcms_apply_map needs scratch (the fields rearranged
// into the operator's source order and a staging copy of the result) and takes it from the
// stream-ordered pool. This entry point uses one file-scope device array instead, of
// NOALLOC_SCRATCH_BYTES, which is part of the loaded library: every GPU that loads the
// library holds it until the process exits, and the entry point itself allocates nothing.
#include <mutex>
#include <string>

#include "pcms_internal.cuh"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB

static __device__ __align__(256) unsigned char g_apply_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_addr[64] = {};   // device address of g_apply_scratch per device ordinal

pcms_status fail_with(pcms_status st, const std::string& msg) {
    pcms::set_last_error_message("pcms_apply_map_noalloc: " + msg);
    return st;
}

}  // namespace

extern "C" pcms_status pcms_apply_map_noalloc(pcms_map map, const void* fields, int n_fields,
                                              void* out, void* stream) {
    if (!map) return fail_with(PCMS_ERR_INVALID_ARG, "map is NULL");
    if (n_fields < 1 || n_fields > 16)
        return fail_with(PCMS_ERR_INVALID_ARG, "n_fields must be in 1..16");
    const pcms::MapImpl& M = map->impl;
    if (M.ns > 0 && !fields) return fail_with(PCMS_ERR_INVALID_ARG, "fields is NULL");
    if (M.nt > 0 && !out) return fail_with(PCMS_ERR_INVALID_ARG, "out is NULL");
    const int64_t need = pcms::apply_scratch_bytes(M, n_fields);
    if (need > (int64_t)NOALLOC_SCRATCH_BYTES)
        return fail_with(PCMS_ERR_CAPACITY,
                         "this map and field count need " + std::to_string(need) +
                             " bytes of scratch, above the fixed " +
                             std::to_string(NOALLOC_SCRATCH_BYTES) +
                             " bytes; use pcms_apply_map");
    // An error left pending on this thread by earlier, unrelated work would surface at this
    // call's first launch check and be reported as this call's own. Leave it pending for its
    // owner, launch nothing, and say so.
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return fail_with(PCMS_ERR_CUDA,
                         std::string("a CUDA error from earlier work is pending on this thread (") +
                             cudaGetErrorString(pending) + "); nothing was launched");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail_with(PCMS_ERR_CUDA, "no usable current device");
    }
    void* scratch = nullptr;
    {
        // Set-up, once per device, with that device current: in host code the array's name
        // stands for a host-side shadow, not a device address, so ask the runtime for it.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return fail_with(PCMS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                                    cudaGetErrorString(e));
            }
            g_addr[dev] = p;
        }
        scratch = g_addr[dev];
    }
    const char* where = "";
    const cudaError_t e = pcms::mls_apply_with_scratch(M, fields, n_fields, out, scratch,
                                                       (cudaStream_t)stream, &where);
    if (e != cudaSuccess)
        return fail_with(PCMS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    pcms::set_last_error_message("");
    return PCMS_OK;
}
