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
// The bounded wait of the TMA-staged kernels, a test hook (environment
// variable LBM_TMA_WAIT_POLLS=<n> when a lattice's staging is set up or a batch
// is created): each tile's wait for its staged copy gives up after n polls of
// the mbarrier instead of the default 2^20, so that n = 0 exercises the
// give-up path (the CTA stops, drains its copy, raises the error flag) without
// any copy failing.  Returns -1 (the default) when unset or not a number >= 0.
inline int tma_wait_polls() {
    const char* c = std::getenv("LBM_TMA_WAIT_POLLS");
    if (!c || !*c) return -1;
    char* end = nullptr;
    const long v = std::strtol(c, &end, 10);
    return (*end == '\0' && v >= 0 && v <= (1l << 30)) ? static_cast<int>(v) : -1;
}

// `rows` rows of `pitch` elements of `elem` bytes from `buf`, back to back.
inline cudaError_t paint_canary(void* buf, size_t elem, long long nx, long long pitch,
                                long long rows, cudaStream_t st) {
    if (pitch <= nx) return cudaSuccess;
    return cudaMemset2DAsync(static_cast<char*>(buf) + nx * elem, pitch * elem, 0xFF,
                             (pitch - nx) * elem, static_cast<size_t>(rows), st);
}

}  // namespace lbm
