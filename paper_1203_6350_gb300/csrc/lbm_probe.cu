// Bandwidth probe for the roofline denominators (not part of the scheme).
//
// One launch copies a buffer into another and back, `iters` times, without
// launch gaps: each thread owns the 16-byte words t, t + T, t + 2T, ... (T the
// number of threads in the grid, so neighbouring threads touch neighbouring
// words) and copies the same words in both directions, so no thread ever waits
// for another and no barrier is needed.  With both buffers inside L2 this measures the
// L2-resident copy rate over that working set; larger than L2, the HBM copy
// rate.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm.h"

namespace {

__global__ void __launch_bounds__(512) probe_copy_kernel(uint4* __restrict__ a,
                                                         uint4* __restrict__ b,
                                                         long long words, int iters) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    const long long first = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int k = 0; k < iters; ++k) {
        const uint4* src = (k & 1) ? b : a;
        uint4* dst = (k & 1) ? a : b;
        for (long long i = first; i < words; i += stride) dst[i] = src[i];
    }
}

}  // namespace

extern "C" int lbm_probe_copy(void* a, void* b, size_t bytes, int iters, void* cuda_stream) {
    if (!a || !b || bytes < 16 || bytes % 16 != 0 || iters < 1) return LBM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) % 16 != 0)
        return LBM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ERR_CUDA;
    const long long words = static_cast<long long>(bytes / 16);
    probe_copy_kernel<<<4 * sms, 512, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        static_cast<uint4*>(a), static_cast<uint4*>(b), words, iters);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
