// pcms_batch.cuh -- the batched one-shot MLS transfer of many small problems (batch.cu):
// the device table the two batch kernels read, and the host executor that fills it and
// launches (or replays, as one CUDA graph per shape class) the kernels.
#pragma once

#include <string>
#include <vector>

#include "pcms_internal.cuh"

namespace pcms {

// shape classes: (dim - 2) * 6 + basis_degree * 2 + (32 lanes per target ? 1 : 0)
constexpr int BATCH_CLASSES = 12;

// Per-class header of the device table: the work counter of k_batch_mls (reset by
// k_batch_sort) and the per-problem error flags (1 = a non-finite coordinate).
struct BatchHeader {
    int n_req;
    int pad_;
    long long total_tiles;
    unsigned long long next;
    // targets whose FP64 normal equations are too ill-conditioned for the bound, solved
    // again by Householder QR (k_batch_qr): (problem, target) pairs, count and capacity
    int2* qr_list;
    unsigned int n_qr;
    unsigned int qr_cap;
    int32_t err[PCMS_BATCH_MAX_ITEMS];
};

// One problem of a batch. Caller buffers and the problem's part of the batch's scratch
// arena are filled on the host; the grid (lo, h, inv_h, n, rcell) by k_batch_sort.
struct BatchReq {
    const double* src;      // [dim][ns] (caller order)
    const double* tgt;      // [dim][nt]
    const float* fields;    // [nf][ns]
    float* out;             // [nf][nt]
    int8_t* status;         // [nt] or null
    int32_t* cell_start;    // [cap_cells + 1]: counts, then cell starts
    int32_t* cursor;        // [cap_cells] scatter cursors
    int32_t* keys;          // [ns] cell of each source
    int32_t* perm;          // [ns] sorted position -> source index
    double* x64;            // [dim][ns] sorted FP64 coordinates
    float4* hl0;            // [ns] sorted FP32 hi/lo offsets from lo (2D {xh,yh,xl,yl};
    float2* hl1;            //      3D {xh,yh,zh,xl} and {yl,zl})
    float* fs;              // [ns][fp] fields in sorted order, zero-padded
    int64_t ns, nt, cap_cells;
    long long tile0;        // the problem's first work unit
    double radius, r2, inv_r;
    float r2f, inv_rf;
    int nf, fp, weight, pad_;
    double lo[3];
    double h, inv_h;
    int n[3];
    float rcell;
};

int batch_class_of(const pcms_batch_item& it);
int64_t batch_item_bytes(const pcms_batch_item& it);   // device scratch of one item
std::string batch_check_item(const pcms_batch_item& it);   // "" if the item is valid

// Runs batches on a caller's stream. With use_graphs, each shape class's table copy and
// kernels are captured once into a CUDA graph (from page-locked table memory) and replayed
// for every later batch of that class on the same executor; the executor is then used by
// one thread at a time. run() returns after enqueueing; with `result` it syncs the stream
// once and writes each item's status. A graph executor always needs `result` (its
// page-locked table may only be rewritten after the stream has passed the copy).
class BatchExec {
public:
    explicit BatchExec(bool use_graphs);
    ~BatchExec();
    BatchExec(const BatchExec&) = delete;
    BatchExec& operator=(const BatchExec&) = delete;
    void run(const pcms_batch_item* items, int n, int32_t* result, cudaStream_t s);

private:
    void capture(int c, void* td, const void* th, size_t bytes, BatchHeader* hdr_d, BatchReq* req_d,
                 cudaStream_t s);
    bool graphs_;
    bool no_graph_[BATCH_CLASSES] = {};
    void* table_d_ = nullptr;
    void* table_h_ = nullptr;
    int32_t* err_h_ = nullptr;
    std::vector<char> table_v_;
    std::vector<int32_t> err_v_;
    cudaGraphExec_t exec_[BATCH_CLASSES] = {};
};

}  // namespace pcms
