// tune.cu -- the plan tuning table: per (dimension, basis degree, precision, mode, bucket)
// the lanes per target and the grid's cell divisor that a measurement found fastest, and per
// field count the apply form (pcms_tune_set; the Python tuner measures and writes it). The
// plan rules of mls.cu consult it; without an entry they stand. Readers take a snapshot of
// the table (a shared pointer), so it can be replaced while requests run.
#include <atomic>
#include <cmath>
#include <memory>
#include <mutex>
#include <vector>

#include "pcms_internal.cuh"

namespace pcms {

std::mutex g_mu;
std::shared_ptr<const std::vector<TuneEntry>> g_table;

std::shared_ptr<const std::vector<TuneEntry>> snapshot() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_table;
}

int tune_bucket(double mean) {
    if (!(mean >= 1.0)) return 0;
    return std::min(30, (int)std::floor(std::log2(mean)));
}

bool tune_lookup(int dim, int degree, bool mixed, int mode, int bucket, TuneEntry* out) {
    const auto t = snapshot();
    if (!t) return false;
    for (const TuneEntry& e : *t) {
        if (e.dim == dim && e.degree == degree && e.mixed == (int)mixed && e.mode == mode &&
            e.bucket == bucket) {
            *out = e;
            return true;
        }
    }
    return false;
}

}  // namespace pcms

extern "C" {

pcms_status pcms_tune_set(const pcms_tune_entry* entries, int n) {
    if (n < 0 || (n > 0 && !entries)) return PCMS_ERR_INVALID_ARG;
    auto t = std::make_shared<std::vector<pcms::TuneEntry>>();
    for (int i = 0; i < n; i++) {
        const pcms_tune_entry& e = entries[i];
        const bool apply = e.mode == PCMS_TUNE_APPLY;
        if (e.dim < 2 || e.dim > 3 || e.degree < 0 || e.degree > 2 ||
            (e.precision != PCMS_FP64 && e.precision != PCMS_MIXED) ||
            (e.mode != PCMS_TUNE_MAP && e.mode != PCMS_TUNE_ONESHOT && !apply) || e.bucket < 0 ||
            (!apply && e.lanes != 8 && e.lanes != 32) ||
            (!apply && !(e.cell_div >= 1.0 && e.cell_div <= 8.0)) ||
            (apply && (e.apply_form < 0 || e.apply_form > 1 || e.bucket < 1 || e.bucket > 16)))
            return PCMS_ERR_INVALID_ARG;
        pcms::TuneEntry x;
        x.dim = e.dim;
        x.degree = e.degree;
        x.mixed = e.precision == PCMS_MIXED;
        // the library's own mode numbers: 1 = operator (map), 2 = one-shot, 3 = apply
        x.mode = e.mode;
        x.bucket = e.bucket;
        x.lanes = e.lanes;
        x.cell_div = e.cell_div;
        x.apply_form = e.apply_form;
        t->push_back(x);
    }
    std::lock_guard<std::mutex> lk(pcms::g_mu);
    pcms::g_table = n > 0 ? std::shared_ptr<const std::vector<pcms::TuneEntry>>(std::move(t)) : nullptr;
    return PCMS_OK;
}

int pcms_tune_count(void) {
    const auto t = pcms::snapshot();
    return t ? (int)t->size() : 0;
}

pcms_status pcms_tune_get(int i, pcms_tune_entry* out) {
    const auto t = pcms::snapshot();
    if (!out || !t || i < 0 || i >= (int)t->size()) return PCMS_ERR_INVALID_ARG;
    const pcms::TuneEntry& x = (*t)[(size_t)i];
    out->dim = x.dim;
    out->degree = x.degree;
    out->precision = x.mixed ? PCMS_MIXED : PCMS_FP64;
    out->mode = x.mode;
    out->bucket = x.bucket;
    out->lanes = x.lanes;
    out->cell_div = x.cell_div;
    out->apply_form = x.apply_form;
    return PCMS_OK;
}

}  // extern "C"
