// Test kernel: applies the library's device FP64 reciprocal (pcms::recip64, Newton-Raphson
// from the FP32 reciprocal) to an array, for comparison with IEEE division on the host.
#include "pcms_internal.cuh"

namespace {
__global__ void k_recip64(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = pcms::recip64(x[i]);
}
}  // namespace

extern "C" int recip64_run(const double* x, double* y, int64_t n, void* stream) {
    if (n <= 0) return 0;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_recip64<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, y, n);
    return (int)cudaGetLastError();
}
