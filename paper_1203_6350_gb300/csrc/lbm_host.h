// Host-side helpers of the C-ABI layer (no kernels): NVTX ranges over API
// calls and the padding canaries.  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdlib>
#include <cstring>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace lbm {

// An NVTX range over one API call, so that profilers can group its launches
// (e.g. ncu --nvtx --nvtx-include "lbm_step/").  Without a tool attached a
// push or pop is one check of a function pointer.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Padding canaries, a debugging aid (environment variable LBM_CANARY=1 when a
// lattice, batch or 3-D lattice is created): the padding of every row --
// elements [nx, pitch) -- of every plane of both population buffers is filled
// with all-one bytes, a NaN in each storage format.  No kernel reads or writes
// padding, so a stray read shows up as NaN in the results and a stray write as
// a changed canary in the raw state.
inline bool canary_requested() {
    const char* c = std::getenv("LBM_CANARY");
    return c && !std::strcmp(c, "1");
}
// `rows` rows of `pitch` elements of `elem` bytes from `buf`, back to back.
inline cudaError_t paint_canary(void* buf, size_t elem, long long nx, long long pitch,
                                long long rows, cudaStream_t st) {
    if (pitch <= nx) return cudaSuccess;
    return cudaMemset2DAsync(static_cast<char*>(buf) + nx * elem, pitch * elem, 0xFF,
                             (pitch - nx) * elem, static_cast<size_t>(rows), st);
}

}  // namespace lbm
