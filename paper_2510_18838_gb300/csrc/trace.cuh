// trace.cuh -- scope object that times one kernel launch with CUDA events on its stream
// (or only counts it) when tracing is enabled (pcms_trace_enable).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pcms {

bool trace_on();       // mode 1 or 2
bool trace_timing();   // mode 1: events, and work counts that cost extra launches
void trace_enable(int mode);
// record a count (not a launch) under "count:<name>" while tracing is on
void trace_count(const char* name, int64_t n);
int trace_count();
int trace_get(int i, char* name, int name_len, int64_t* launches, double* total_ms);

class TraceScope {
public:
    TraceScope(const char* name, cudaStream_t s);
    ~TraceScope();
    TraceScope(const TraceScope&) = delete;
    TraceScope& operator=(const TraceScope&) = delete;

private:
    const char* name_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr;
};

}  // namespace pcms

#define PCMS_TRACE_CAT2(a, b) a##b
#define PCMS_TRACE_CAT(a, b) PCMS_TRACE_CAT2(a, b)
#define PCMS_TRACE(name, stream) ::pcms::TraceScope PCMS_TRACE_CAT(pcms_trace_, __LINE__)(name, stream)
