// serve.cu -- continuous-batching request loop around the transfer kernels.
//
// n_slots worker threads each own a non-blocking CUDA stream. Requests are admitted in
// submission order when a slot is idle and their device-memory estimate fits under the
// cap together with what is already admitted or cached; cached operators that no running
// request uses are evicted least-recently-used first. Each admitted request runs entirely
// on its slot's stream (the library's own syncs wait for that stream only), so requests on
// different slots overlap on the GPU. Completion is taken after the slot's stream has
// drained. No thread ever waits on the GPU without a bounded host-side timeout path: the
// client's drain/poll calls have explicit timeouts.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pcms_batch.cuh"
#include "pcms_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    pcms_request req;
    int64_t ticket = 0;
    int64_t bytes = 0;
    double t_submit = 0, t_start = 0, t_end = 0;
    pcms_status st = PCMS_OK;
    int used_cached = 0;
    bool builds_cache = false;
};

// Page-locked bounce buffers of one slot: host-I/O requests whose buffers are ordinary
// (pageable) memory are copied through them in chunks, the slot's thread copying one chunk
// on the CPU while the GPU transfers the other. Allocated on first use.
constexpr size_t BOUNCE_BYTES = size_t(16) << 20;
struct Bounce {
    char* h[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    int cur = 0;
};

struct CacheEntry {
    std::unique_ptr<pcms::MapImpl> map;
    int64_t bytes = 0;       // bytes charged to the cap while cached
    bool ready = false;
    int pins = 0;
    uint64_t last_use = 0;
};

}  // namespace

struct pcms_server_s {
    int device = 0;
    int n_slots = 1;
    int64_t cap = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_cache;
    std::deque<Job*> queue;
    std::vector<std::unique_ptr<Job>> jobs;
    std::deque<int64_t> finished;
    int64_t n_submitted = 0, n_completed = 0;
    int64_t in_use = 0, peak = 0;
    uint64_t use_clock = 0;
    bool stop = false;
    std::unordered_map<int64_t, CacheEntry> cache;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::vector<Bounce> bounce;   // per slot
    // batched small MLS requests (batch.cu): requests with at most batch_max points per
    // set go through one graph replay per shape class with the other queued ones; 0 = off
    int64_t batch_max = 8192;
    std::vector<std::unique_ptr<pcms::BatchExec>> batch;   // per slot, made by its worker
    int64_t n_batches = 0, n_batched = 0;

    double now() const {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
};

namespace {

int64_t mls_elem(const pcms_request& r) { return r.opts.precision == PCMS_MIXED ? 4 : 8; }

// bytes of the request's buffers when the server stages them (host_io): geometry, and
// fields/outputs; `geometry` false for an apply of a cached operator
int64_t staged_bytes(const pcms_request& r, bool geometry) {
    if (!r.host_io) return 0;
    if (r.kind == PCMS_REQ_MESH)
        return 16 * r.n_src + 12 * r.n_tri + 16 * r.n_tgt + 4 * r.n_tgt +
               (r.out ? 8 * (r.n_src + r.n_tgt) : 0) + 6 * 256;
    const int64_t f = (int64_t)std::max(r.n_fields, 1) * mls_elem(r) * (r.n_src + r.n_tgt);
    return f + (geometry ? 8LL * r.dim * (r.n_src + r.n_tgt) : 0) + 4 * 256;
}

int64_t request_bytes(const pcms_request& r) {
    if (r.bytes_hint > 0) return r.bytes_hint;
    if (r.kind == PCMS_REQ_MESH)
        return pcms::estimate_mesh_bytes(r.n_src, r.n_tri, r.n_tgt) + staged_bytes(r, true);
    pcms::MlsParams P = pcms::make_mls_params(r.dim, r.basis_degree, r.radius, r.opts);
    const bool keep = r.map_key >= 0;
    return pcms::estimate_mls_bytes(P, r.n_src, r.n_tgt, r.n_fields, keep) +
           staged_bytes(r, true);
}

// A request the batched path takes: a one-shot mixed MLS transfer (no operator kept or
// reused) with the user's radius, lambda = 0, and at most batch_max points per set.
bool batchable(const pcms_server_s* S, const pcms_request& r) {
    return S->batch_max > 0 && r.kind == PCMS_REQ_MLS && !r.reuse_map && r.map_key < 0 &&
           r.opts.precision == PCMS_MIXED && r.opts.min_neighbors == 0 && r.opts.lambda == 0.0 &&
           (r.dim == 2 || r.dim == 3) && r.n_src <= S->batch_max && r.n_tgt <= S->batch_max &&
           r.n_src <= PCMS_BATCH_MAX_POINTS && r.n_tgt <= PCMS_BATCH_MAX_POINTS;
}

pcms_batch_item batch_item(const pcms_request& r) {
    pcms_batch_item it{};
    it.dim = r.dim;
    it.basis_degree = r.basis_degree;
    it.radius = r.radius;
    it.weight = r.opts.weight;
    it.src_pts = r.src_pts;
    it.n_src = r.n_src;
    it.tgt_pts = r.tgt_pts;
    it.n_tgt = r.n_tgt;
    it.fields = (const float*)r.fields;
    it.n_fields = r.n_fields;
    it.out = (float*)r.out;
    it.target_status = nullptr;
    return it;
}

bool page_locked(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

void bounce_init(Bounce& b) {
    if (b.h[0]) return;
    for (int i = 0; i < 2; i++) {
        PCMS_CU(cudaHostAlloc((void**)&b.h[i], BOUNCE_BYTES, cudaHostAllocDefault));
        PCMS_CU(cudaEventCreateWithFlags(&b.ev[i], cudaEventDisableTiming));
    }
}

// host -> device on stream s: directly from page-locked memory, else through the bounce
// buffers (the CPU fills one while the GPU reads the other)
void copy_in(Bounce& b, void* dst, const void* src, size_t n, cudaStream_t s) {
    if (page_locked(src)) {
        PCMS_CU(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s));
        return;
    }
    bounce_init(b);
    for (size_t off = 0; off < n; off += BOUNCE_BYTES) {
        const size_t len = std::min(BOUNCE_BYTES, n - off);
        const int c = b.cur;
        if (b.used[c]) PCMS_CU(cudaEventSynchronize(b.ev[c]));
        std::memcpy(b.h[c], (const char*)src + off, len);
        PCMS_CU(cudaMemcpyAsync((char*)dst + off, b.h[c], len, cudaMemcpyHostToDevice, s));
        PCMS_CU(cudaEventRecord(b.ev[c], s));
        b.used[c] = true;
        b.cur = c ^ 1;
    }
}

// device -> host after the work queued on s: chunk k is transferred while chunk k-1 is
// copied out of the other buffer
void copy_out(Bounce& b, void* dst, const void* src, size_t n, cudaStream_t s) {
    if (page_locked(dst)) {
        PCMS_CU(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s));
        return;
    }
    bounce_init(b);
    int cp = -1;
    size_t op = 0, lp = 0;
    for (size_t off = 0; off < n; off += BOUNCE_BYTES) {
        const size_t len = std::min(BOUNCE_BYTES, n - off);
        const int c = b.cur;
        if (b.used[c]) PCMS_CU(cudaEventSynchronize(b.ev[c]));
        PCMS_CU(cudaMemcpyAsync(b.h[c], (const char*)src + off, len, cudaMemcpyDeviceToHost, s));
        PCMS_CU(cudaEventRecord(b.ev[c], s));
        b.used[c] = true;
        if (cp >= 0) {
            PCMS_CU(cudaEventSynchronize(b.ev[cp]));
            std::memcpy((char*)dst + op, b.h[cp], lp);
        }
        cp = c;
        op = off;
        lp = len;
        b.cur = c ^ 1;
    }
    if (cp >= 0) {
        PCMS_CU(cudaEventSynchronize(b.ev[cp]));
        std::memcpy((char*)dst + op, b.h[cp], lp);
    }
}

// Device staging of a host_io request: copies in, on the slot's stream, what the chosen
// path reads; outputs are copied back by unstage().
struct Staging {
    pcms::DBuf buf;
    char* next = nullptr;
    Bounce* bounce = nullptr;
    pcms_request d;   // the request with device pointers
    const void* take(const void* host, int64_t bytes, cudaStream_t s) {
        if (!host || bytes <= 0) return nullptr;
        void* p = next;
        next += (bytes + 255) / 256 * 256;
        copy_in(*bounce, p, host, (size_t)bytes, s);
        return p;
    }
    void* room(const void* host, int64_t bytes) {
        if (!host || bytes <= 0) return nullptr;
        void* p = next;
        next += (bytes + 255) / 256 * 256;
        return p;
    }
};

void stage(const pcms_request& r, bool geometry, Staging& st, cudaStream_t s) {
    st.d = r;
    st.buf.alloc((size_t)staged_bytes(r, geometry), s);
    st.next = (char*)st.buf.p;
    if (r.kind == PCMS_REQ_MESH) {
        st.d.src_pts = (const double*)st.take(r.src_pts, 16 * r.n_src, s);
        st.d.tri = (const int32_t*)st.take(r.tri, 12 * r.n_tri, s);
        st.d.tgt_pts = (const double*)st.take(r.tgt_pts, 16 * r.n_tgt, s);
        st.d.fields = r.out ? st.take(r.fields, 8 * r.n_src, s) : nullptr;
        st.d.out = st.room(r.out, 8 * r.n_tgt);
        st.d.elem_ids = (int32_t*)st.room(r.elem_ids, 4 * r.n_tgt);
        return;
    }
    const int64_t e = mls_elem(r);
    if (geometry) {
        st.d.src_pts = (const double*)st.take(r.src_pts, 8LL * r.dim * r.n_src, s);
        st.d.tgt_pts = (const double*)st.take(r.tgt_pts, 8LL * r.dim * r.n_tgt, s);
    }
    st.d.fields = st.take(r.fields, (int64_t)r.n_fields * e * r.n_src, s);
    st.d.out = st.room(r.out, (int64_t)r.n_fields * e * r.n_tgt);
}

void unstage(const pcms_request& r, const Staging& st, cudaStream_t s) {
    if (r.kind == PCMS_REQ_MESH) {
        if (r.out) copy_out(*st.bounce, r.out, st.d.out, 8 * r.n_tgt, s);
        copy_out(*st.bounce, r.elem_ids, st.d.elem_ids, 4 * r.n_tgt, s);
        return;
    }
    copy_out(*st.bounce, r.out, st.d.out, (size_t)r.n_fields * mls_elem(r) * r.n_tgt, s);
}

// evict unpinned cached operators (LRU) until `need` more bytes fit; caller holds the lock
void evict_for(pcms_server_s* S, int64_t need) {
    while (S->in_use + need > S->cap) {
        auto victim = S->cache.end();
        for (auto it = S->cache.begin(); it != S->cache.end(); ++it) {
            if (!it->second.ready || it->second.pins > 0) continue;
            if (victim == S->cache.end() || it->second.last_use < victim->second.last_use) victim = it;
        }
        if (victim == S->cache.end()) return;
        S->in_use -= victim->second.bytes;
        S->cache.erase(victim);   // frees the operator on the stream that built it
    }
}

void run_job(pcms_server_s* S, Job* j, cudaStream_t s, Bounce& bounce, pcms::MapImpl* cached,
             std::unique_ptr<pcms::MapImpl>* built) {
    Staging st;
    st.bounce = &bounce;
    if (j->req.host_io) stage(j->req, cached == nullptr, st, s);
    const pcms_request& r = j->req.host_io ? st.d : j->req;
    if (r.kind == PCMS_REQ_MESH) {
        pcms::MeshImpl mesh;
        mesh.stream = s;
        pcms::mesh_create(mesh, r.src_pts, r.n_src, r.tri, r.n_tri);
        pcms::mesh_locate(mesh, r.tgt_pts, r.n_tgt, r.out ? (const double*)r.fields : nullptr,
                          r.elem_ids, nullptr, (double*)r.out, s);
        if (j->req.host_io) unstage(j->req, st, s);
        PCMS_CU(cudaStreamSynchronize(s));
        return;
    }
    pcms::MlsParams P = pcms::make_mls_params(r.dim, r.basis_degree, r.radius, r.opts);
    if (cached) {
        // the operator's sizes bound every access of the apply: they must be the request's
        if (cached->ns != r.n_src || cached->nt != r.n_tgt || cached->P.dim != r.dim ||
            cached->P.prec != r.opts.precision)
            pcms::fail(PCMS_ERR_INVALID_ARG,
                       "reuse_map: the cached operator under this map_key has other sizes");
        pcms::mls_apply(*cached, r.fields, r.n_fields, r.out, s);
    } else if (built) {
        std::unique_ptr<pcms::MapImpl> M(new pcms::MapImpl());
        M->P = P;
        M->ns = r.n_src;
        M->nt = r.n_tgt;
        M->stream = s;
        pcms::mls_create_map(*M, r.src_pts, r.tgt_pts, r.opts);
        pcms::mls_apply(*M, r.fields, r.n_fields, r.out, s);
        *built = std::move(M);
    } else if (r.n_fields <= 2 || r.opts.precision == PCMS_MIXED) {
        // one-shot: fused walks for one or two fields, else the operator's rows applied as
        // they are evaluated (mixed)
        int64_t nu = 0;
        pcms::mls_transfer(P, r.src_pts, r.n_src, r.tgt_pts, r.n_tgt, r.opts, r.fields,
                           r.n_fields, r.out, nullptr, s, &nu);
    } else {
        pcms::MapImpl M;
        M.P = P;
        M.ns = r.n_src;
        M.nt = r.n_tgt;
        M.stream = s;
        pcms::mls_create_map(M, r.src_pts, r.tgt_pts, r.opts);
        pcms::mls_apply(M, r.fields, r.n_fields, r.out, s);
    }
    if (j->req.host_io) unstage(j->req, st, s);
    PCMS_CU(cudaStreamSynchronize(s));
}

// Device bytes of a request on the batched path: its part of the batch's scratch arena and
// its staged copies, plus 64 KiB for the batch's table and rounding.
int64_t batch_bytes(const pcms_request& r) {
    return pcms::batch_item_bytes(batch_item(r)) + staged_bytes(r, true) + (int64_t(1) << 16);
}

// Targets of one batch at most: bounds a batch's time, so that requests queued behind it
// wait for a few milliseconds at most.
constexpr int64_t BATCH_MAX_TARGETS = int64_t(1) << 21;

// With the lock held and the head request batchable: take the head and the other queued
// batchable requests that fit under the cap (at most PCMS_BATCH_MAX_ITEMS, at most
// BATCH_MAX_TARGETS targets), in queue order, off the queue. Empty if the head does not fit.
std::vector<Job*> take_batch(pcms_server_s* S) {
    std::vector<Job*> b;
    int64_t need = 0, targets = 0;
    const int64_t head = batch_bytes(S->queue.front()->req);
    if (S->in_use + head > S->cap) evict_for(S, head);
    for (Job* x : S->queue) {
        if ((int)b.size() >= PCMS_BATCH_MAX_ITEMS) break;
        if (!batchable(S, x->req)) continue;
        const int64_t xb = batch_bytes(x->req);
        if (S->in_use + need + xb > S->cap) break;
        if (!b.empty() && targets + x->req.n_tgt > BATCH_MAX_TARGETS) break;
        b.push_back(x);
        need += xb;
        targets += x->req.n_tgt;
        x->bytes = xb;
    }
    if (b.empty()) return b;
    std::deque<Job*> rest;
    size_t k = 0;
    for (Job* x : S->queue) {
        if (k < b.size() && x == b[k]) k++;
        else rest.push_back(x);
    }
    S->queue.swap(rest);
    S->in_use += need;
    S->peak = std::max(S->peak, S->in_use);
    const double t = S->now();
    for (Job* x : b) x->t_start = t;
    S->n_batches++;
    S->n_batched += (int64_t)b.size();
    return b;
}

// Runs a batch on the slot's stream (staging host-I/O requests' buffers) and completes its
// requests.
void run_batch(pcms_server_s* S, const std::vector<Job*>& b, int slot) {
    cudaStream_t s = S->streams[slot];
    std::vector<pcms_status> st(b.size(), PCMS_OK);
    try {
        if (!S->batch[slot]) S->batch[slot].reset(new pcms::BatchExec(true));
        std::vector<Staging> stg(b.size());
        std::vector<pcms_batch_item> items(b.size());
        for (size_t i = 0; i < b.size(); i++) {
            const pcms_request& r = b[i]->req;
            if (r.host_io) {
                stg[i].bounce = &S->bounce[slot];
                stage(r, true, stg[i], s);
                items[i] = batch_item(stg[i].d);
            } else {
                items[i] = batch_item(r);
            }
        }
        std::vector<int32_t> res(b.size(), PCMS_OK);
        S->batch[slot]->run(items.data(), (int)items.size(), res.data(), s);
        for (size_t i = 0; i < b.size(); i++) {
            st[i] = (pcms_status)res[i];
            if (b[i]->req.host_io && st[i] == PCMS_OK) unstage(b[i]->req, stg[i], s);
        }
        PCMS_CU(cudaStreamSynchronize(s));
    } catch (const pcms::PcmsError& e) {
        if (e.status == PCMS_ERR_CUDA)
            std::fprintf(stderr, "pcms server: a batch of %zu requests failed: %s\n", b.size(),
                         e.msg.c_str());
        for (auto& x : st) x = e.status;
    } catch (...) {
        for (auto& x : st) x = PCMS_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        const double t = S->now();
        for (size_t i = 0; i < b.size(); i++) {
            b[i]->st = st[i];
            b[i]->t_end = t;
            S->in_use -= b[i]->bytes;
            S->finished.push_back(b[i]->ticket);
            S->n_completed++;
        }
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

void worker(pcms_server_s* S, int slot) {
    cudaSetDevice(S->device);
    cudaStream_t s = S->streams[slot];
    for (;;) {
        Job* j = nullptr;
        pcms::MapImpl* cached = nullptr;
        std::vector<Job*> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop && S->queue.empty()) return;
                if (!S->queue.empty()) {
                    Job* h = S->queue.front();
                    if (h->bytes > S->cap) {   // can never fit
                        S->queue.pop_front();
                        h->st = PCMS_ERR_CAPACITY;
                        h->t_start = h->t_end = S->now();
                        S->finished.push_back(h->ticket);
                        S->n_completed++;
                        S->cv_done.notify_all();
                        continue;
                    }
                    if (batchable(S, h->req)) {
                        batch = take_batch(S);
                        if (!batch.empty()) break;
                        S->cv_work.wait(lk);
                        continue;
                    }
                    // a reuse request whose operator is being built waits for it
                    const pcms_request& r = h->req;
                    int64_t need = h->bytes;
                    bool reuse = r.kind == PCMS_REQ_MLS && r.reuse_map && r.map_key >= 0;
                    auto it = reuse ? S->cache.find(r.map_key) : S->cache.end();
                    if (reuse && it != S->cache.end() && !it->second.ready) {
                        S->cv_cache.wait(lk);
                        continue;
                    }
                    const bool hit = reuse && it != S->cache.end();
                    if (hit) {
                        // only the apply scratch (fields padded to the vector width, as the
                        // apply allocates it) and the staged fields are new
                        need = pcms::apply_scratch_bytes(*it->second.map, std::max(r.n_fields, 1)) +
                               (int64_t(1) << 20) + staged_bytes(r, false);
                        // pinned across the eviction below: evicting the operator this request
                        // is about to use would leave `it` (and the operator) freed
                        it->second.pins++;
                    }
                    if (S->in_use + need > S->cap) evict_for(S, need);
                    if (hit && S->in_use + need > S->cap) {   // not admitted
                        it->second.pins--;
                        if (it->second.pins == 0) {
                            // no room beside its own operator, which no one else is using:
                            // drop it, and the request (it carries its geometry) builds it again
                            S->in_use -= it->second.bytes;
                            S->cache.erase(it);
                            continue;
                        }
                    }
                    if (S->in_use + need <= S->cap) {
                        S->queue.pop_front();
                        h->bytes = need;
                        S->in_use += need;
                        S->peak = std::max(S->peak, S->in_use);
                        h->t_start = S->now();
                        if (hit) {   // already pinned above
                            it->second.last_use = ++S->use_clock;
                            cached = it->second.map.get();
                            h->used_cached = 1;
                        } else if (r.kind == PCMS_REQ_MLS && r.map_key >= 0 &&
                                   S->cache.find(r.map_key) == S->cache.end()) {
                            CacheEntry e;
                            e.ready = false;
                            S->cache.emplace(r.map_key, std::move(e));
                            h->builds_cache = true;
                        }
                        j = h;
                        break;
                    }
                }
                S->cv_work.wait(lk);
            }
        }
        if (!batch.empty()) {
            run_batch(S, batch, slot);
            continue;
        }
        std::unique_ptr<pcms::MapImpl> built;
        pcms_status st = PCMS_OK;
        try {
            run_job(S, j, s, S->bounce[slot], cached, j->builds_cache ? &built : nullptr);
        } catch (const pcms::PcmsError& e) {
            st = e.status;
            // a CUDA error ends the context for every later request: say where it surfaced
            if (st == PCMS_ERR_CUDA)
                std::fprintf(stderr, "pcms server: request %lld (kind %d, n_src %lld, n_tgt %lld) failed: %s\n",
                             (long long)j->ticket, (int)j->req.kind, (long long)j->req.n_src,
                             (long long)j->req.n_tgt, e.msg.c_str());
        } catch (...) {
            st = PCMS_ERR_CUDA;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            j->st = st;
            j->t_end = S->now();
            S->in_use -= j->bytes;
            if (cached) {
                auto it = S->cache.find(j->req.map_key);
                if (it != S->cache.end()) it->second.pins--;
            }
            if (j->builds_cache) {
                auto it = S->cache.find(j->req.map_key);
                if (st == PCMS_OK && built) {
                    int64_t b = built->device_bytes();
                    it->second.map = std::move(built);
                    it->second.bytes = b;
                    it->second.ready = true;
                    it->second.last_use = ++S->use_clock;
                    S->in_use += b;
                    S->peak = std::max(S->peak, S->in_use);
                    if (S->in_use > S->cap) evict_for(S, 0);
                } else if (it != S->cache.end()) {
                    S->cache.erase(it);
                }
                S->cv_cache.notify_all();
            }
            S->finished.push_back(j->ticket);
            S->n_completed++;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

thread_local std::string g_server_err;

}  // namespace

extern "C" {

pcms_status pcms_server_create(int n_slots, int64_t mem_cap_bytes, pcms_server* out) {
    if (!out || n_slots < 1 || n_slots > 64 || mem_cap_bytes <= 0) return PCMS_ERR_INVALID_ARG;
    *out = nullptr;
    pcms_server_s* S = new pcms_server_s();
    S->n_slots = n_slots;
    S->cap = mem_cap_bytes;
    S->t0 = Clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return PCMS_ERR_CUDA;
    }
    pcms::ensure_mempool(S->device);
    for (int i = 0; i < n_slots; i++) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            delete S;
            return PCMS_ERR_CUDA;
        }
        S->streams.push_back(st);
    }
    S->bounce.resize(n_slots);
    S->batch.resize(n_slots);
    for (int i = 0; i < n_slots; i++) S->workers.emplace_back(worker, S, i);
    *out = S;
    return PCMS_OK;
}

pcms_status pcms_server_submit(pcms_server S, const pcms_request* req, int64_t* ticket) {
    if (!S || !req) return PCMS_ERR_INVALID_ARG;
    const pcms_request& r = *req;
    if (r.kind == PCMS_REQ_MLS) {
        if ((r.dim != 2 && r.dim != 3) || r.basis_degree < 0 || r.basis_degree > 2 ||
            !(r.radius > 0.0) || r.n_fields < 1 || r.n_fields > 16 || r.n_src < 0 || r.n_tgt < 0 ||
            (r.n_tgt > 0 && !r.out) || (r.n_src > 0 && !r.fields) ||
            (r.n_src > 0 && !r.src_pts) || (r.n_tgt > 0 && !r.tgt_pts))
            return PCMS_ERR_INVALID_ARG;
    } else if (r.kind == PCMS_REQ_MESH) {
        if (r.n_src < 0 || r.n_tri < 0 || r.n_tgt < 0 || (r.n_src > 0 && !r.src_pts) ||
            (r.n_tri > 0 && !r.tri) || (r.n_tgt > 0 && (!r.tgt_pts || !r.elem_ids)) ||
            (r.out && !r.fields))
            return PCMS_ERR_INVALID_ARG;
    } else {
        return PCMS_ERR_INVALID_ARG;
    }
    std::unique_ptr<Job> j(new Job());
    j->req = r;
    j->bytes = request_bytes(r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        j->ticket = S->n_submitted++;
        j->t_submit = S->now();
        if (ticket) *ticket = j->ticket;
        S->queue.push_back(j.get());
        S->jobs.push_back(std::move(j));
    }
    S->cv_work.notify_one();
    return PCMS_OK;
}

pcms_status pcms_server_poll(pcms_server S, pcms_request_result* res, int max_results,
                             double timeout_s, int* n_results) {
    if (!S || !n_results || (max_results > 0 && !res)) return PCMS_ERR_INVALID_ARG;
    *n_results = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->finished.empty() && timeout_s > 0)
        S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                            [&] { return !S->finished.empty(); });
    int n = 0;
    while (n < max_results && !S->finished.empty()) {
        Job* j = S->jobs[(size_t)S->finished.front()].get();
        S->finished.pop_front();
        pcms_request_result& o = res[n++];
        o.ticket = j->ticket;
        o.status = j->st;
        o.t_submit = j->t_submit;
        o.t_start = j->t_start;
        o.t_end = j->t_end;
        o.bytes_reserved = j->bytes;
        o.used_cached_map = j->used_cached;
    }
    *n_results = n;
    return PCMS_OK;
}

pcms_status pcms_server_drain(pcms_server S, double timeout_s) {
    if (!S) return PCMS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                  [&] { return S->n_completed == S->n_submitted; });
    return ok ? PCMS_OK : PCMS_ERR_TIMEOUT;
}

double pcms_server_now(pcms_server S) { return S ? S->now() : 0.0; }

pcms_status pcms_server_set_batching(pcms_server S, int64_t max_points) {
    if (!S || max_points < 0) return PCMS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->batch_max = std::min<int64_t>(max_points, PCMS_BATCH_MAX_POINTS);
    return PCMS_OK;
}

pcms_status pcms_server_batch_stats(pcms_server S, int64_t* n_batches, int64_t* n_batched) {
    if (!S) return PCMS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (n_batches) *n_batches = S->n_batches;
    if (n_batched) *n_batched = S->n_batched;
    return PCMS_OK;
}

pcms_status pcms_server_memory(pcms_server S, int64_t* in_use, int64_t* peak,
                               int64_t* cached_maps) {
    if (!S) return PCMS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (in_use) *in_use = S->in_use;
    if (peak) *peak = S->peak;
    if (cached_maps) *cached_maps = (int64_t)S->cache.size();
    return PCMS_OK;
}

void pcms_server_destroy(pcms_server S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->cv_cache.notify_all();
    for (std::thread& t : S->workers) t.join();
    S->cache.clear();
    S->batch.clear();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (Bounce& b : S->bounce)
        for (int i = 0; i < 2; i++) {
            if (b.h[i]) cudaFreeHost(b.h[i]);
            if (b.ev[i]) cudaEventDestroy(b.ev[i]);
        }
    delete S;
}

}  // extern "C"
