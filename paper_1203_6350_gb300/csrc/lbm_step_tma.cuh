// Two time steps per launch with the tile's input staged by the Tensor Memory
// Accelerator (Dirichlet boundary; FP32, FP16 or BF16 storage).
//
// Same arithmetic as tb2_tile (lbm_step_tb.cuh), different data movement:
//  - A persistent CTA walks the 64 x 16 tiles t = blockIdx.x + k gridDim.x.
//  - The input of a tile -- the nine planes of the box from (x0 - pad, y0 - 2),
//    everything step one pulls -- arrives as ONE cp.async.bulk.tensor copy
//    into shared memory, completing on an mbarrier.  The tensor map's extent is
//    the lattice (nx x ny x 9 planes), so every element outside it reads as
//    zero: exactly the Dirichlet far-field deviation, with no bounds checks in
//    the pulls.  The box starts 16 bytes left of the tile, the alignment a
//    tiled copy's x coordinate needs: pad = 4 FP32 elements (72 x 20 box) or 8
//    16-bit elements (80 x 20 box).
//  - Step one pulls from the staged box; step two from the R1 ring, as in
//    tb2_tile.  The copy of the next tile is issued as soon as step one has
//    read the box, so it overlaps step two.  Two CTAs of 320 threads per SM
//    (96 KB of shared memory each) overlap one another's waits.
//  - Every wait on the mbarrier gives up after a bounded number of polls
//    (`polls`, kTmaPolls by default); the CTA then agrees (a barrier vote) to
//    stop, waits for its copy in flight with a bound 16 times longer, records
//    the failure in *err and returns.
#pragma once

#include <cuda.h>

#include "lbm_step_tb.cuh"

namespace lbm {

// The staged box for storage type T: from 16 bytes left of the tile to 16
// bytes right of it, rows y0 - 2 .. y0 + 17.
template <typename T>
struct TmaBox {
    static constexpr int pad = 16 / static_cast<int>(sizeof(T));  // 4 (FP32), 8 (16-bit)
    static constexpr int w = kTbW + 2 * pad;                      // 72, 80
    static constexpr int h = kTbH + 4;                            // 20
    static constexpr int plane = w * h;                           // elements per plane
    static constexpr unsigned bytes = 9u * plane * sizeof(T);     // 51,840 / 28,800
    static_assert(bytes % 16 == 0, "the ring behind the box stays 16-byte aligned");
};
constexpr int kTmaPad = TmaBox<float>::pad;  // the FP32 box (the batched kernel's)
constexpr int kTmaW = TmaBox<float>::w;
constexpr int kTmaH = TmaBox<float>::h;
constexpr int kTmaPlane = TmaBox<float>::plane;
constexpr unsigned kTmaBoxBytes = TmaBox<float>::bytes;
constexpr int kTmaPolls = 1 << 20;          // mbarrier polls before a wait gives up
constexpr int kTmaDrainPolls = 16 * kTmaPolls;  // the copy in flight, after a give-up
// 10 warps, two CTAs (96 KB each) per SM: step one's 612 pairs and step
// two's 512 then take two rounds each at 96 % and 80 % use (256 threads need
// three rounds for step one; 384 leave a half-empty second round in both).
constexpr int kTmaThreads = 320;

// Threads and resident CTAs per SM of the single-lattice TMA kernel per format.
// 16-bit: a 28.8 KB box and the 44 KB FP32 ring fit three CTAs per SM; at 256
// threads the collision fits the 85 registers that allows (73 for type II).
// Measured at 4096^2-16384^2 against plain loads: -2.5 % (type III) to +1.6 %
// (type II) with 256 x 3, and 10-15 % slower with 320 x 2, so 16-bit staging
// is available but not the default.
template <typename T>
struct TmaLaunch {
    static constexpr int threads = sizeof(T) == 2 ? 256 : kTmaThreads;
    static constexpr int min_blocks = sizeof(T) == 2 ? 3 : 2;
};

constexpr unsigned kTmaRingBytes = 9u * kR1Plane * sizeof(float);  // R1 ring (tb_smem_bytes)
template <typename T = float>
constexpr size_t tma_smem_bytes() {
    return TmaBox<T>::bytes + kTmaRingBytes + 16;  // box, R1 ring, mbarrier
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arm the barrier for the box's bytes and start its copy at (x, y, plane 0).
template <typename T = float>
__device__ __forceinline__ void tma_box_load(T* dst, const CUtensorMap* map,
                                             unsigned long long* bar, int x, int y) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(TmaBox<T>::bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(0),
        "r"(smem_addr(bar))
        : "memory");
}

// Poll the barrier's phase `parity` at most `polls` times.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          int polls = kTmaPolls) {
    for (int i = 0; i < polls; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <typename T, int VAR>
__global__ void __launch_bounds__(TmaLaunch<T>::threads, TmaLaunch<T>::min_blocks)
    step_tb2_tma_kernel(const __grid_constant__ CUtensorMap src_map, T* __restrict__ dst,
                        int nx, int ny, int pitch, unsigned plane, StepConst<F2> k,
                        const AxisCoef<float>* __restrict__ tx,
                        const AxisCoef<float>* __restrict__ ty, int ntx, int ntiles,
                        int* __restrict__ err, int polls) {
    using B = TmaBox<T>;
    constexpr int NT = TmaLaunch<T>::threads;
    constexpr bool UB = UnbiasedScale<T>::value;
    extern __shared__ __align__(128) unsigned char tma_raw[];
    T* box = reinterpret_cast<T*>(tma_raw);
    float* r1 = reinterpret_cast<float*>(tma_raw + B::bytes);
    auto* bar = reinterpret_cast<unsigned long long*>(tma_raw + B::bytes + kTmaRingBytes);
    const int tid = threadIdx.x;
    if (tid == 0) mbar_init(bar);
    __syncthreads();
    // the previous launch wrote this launch's input
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int G = gridDim.x;
    int t = blockIdx.x;
    if (tid == 0 && t < ntiles)
        tma_box_load<T>(box, &src_map, bar, (t % ntx) * kTbW - B::pad, (t / ntx) * kTbH - 2);
    unsigned parity = 0;
    for (; t < ntiles; t += G) {
        const int x0 = (t % ntx) * kTbW, y0 = (t / ntx) * kTbH;
        const bool ok = mbar_wait(bar, parity, polls);
        parity ^= 1u;
        if (!__syncthreads_and(ok)) {  // the whole CTA stops together
            if (tid == 0) {
                mbar_wait(bar, parity ^ 1u, kTmaDrainPolls);  // the copy in flight
                atomicExch(err, 1);
            }
            return;
        }
        // ---- step 1: time t (staged box) -> time t + 1 on R1 (shared memory) ----
        for (int p = tid; p < kR1Pairs * kR1H; p += NT) {
            const int px = p % kR1Pairs, py = p / kR1Pairs;
            const int x = x0 - 2 + 2 * px, y = y0 - 1 + py;
            F2 v[9];
            pull_pair_interior<T, true>(
                box, B::plane, B::w, static_cast<unsigned>((py + 1) * B::w + B::pad - 2 + 2 * px),
                v);
            const bool row_in = y >= 0 && y < ny;
            const bool keep_a = row_in && x >= 0 && x < nx;
            const bool keep_b = row_in && x + 1 >= 0 && x + 1 < nx;
            collide_lanes<VAR, UB, true>(v, min(max(x, 0), nx - 1), min(max(x + 1, 0), nx - 1),
                                         min(max(y, 0), ny - 1), k, tx, ty);
            if (!(keep_a && keep_b)) {  // lanes outside the lattice hold the wall value 0
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    v[i] = f2(keep_a ? f2_lo(v[i]) : 0.0f, keep_b ? f2_hi(v[i]) : 0.0f);
            }
            store_pair<float>(r1, kR1Plane, static_cast<unsigned>(py * kR1W + 2 * px), v);
        }
        __syncthreads();  // the box is read: the next tile's copy may overwrite it
        if (tid == 0 && t + G < ntiles) {
            const int tn = t + G;
            tma_box_load<T>(box, &src_map, bar, (tn % ntx) * kTbW - B::pad, (tn / ntx) * kTbH - 2);
        }
        // ---- step 2: time t + 1 (R1) -> time t + 2 on the tile (HBM) ----
        for (int p = tid; p < (kTbW / 2) * kTbH; p += NT) {
            const int qx = p % (kTbW / 2), qy = p / (kTbW / 2);
            const int x = x0 + 2 * qx, y = y0 + qy;
            if (x >= nx || y >= ny) continue;
            F2 v[9];
            pull_pair_interior<float, true>(r1, kR1Plane, kR1W,
                                            static_cast<unsigned>((qy + 1) * kR1W + 2 * qx + 2), v);
            collide_pair<VAR, UB, true>(v, x, y, nx, k, tx, ty);
            const unsigned o = static_cast<unsigned>(y * pitch + x);
            if (x + 1 < nx)
                store_pair<T, true>(dst, plane, o, v);
            else
                store_lo<T>(dst, plane, o, v);
        }
        __syncthreads();  // R1 is read
    }
    asm volatile("griddepcontrol.launch_dependents;");
}

// Launch two steps (the buffer behind src_map holds time t, dst receives
// t + 2) on a persistent grid of `grid` CTAs; pdl as for the one-step kernels;
// polls < 0 selects kTmaPolls for each tile's wait.
template <typename T>
inline cudaError_t launch_step_tb2_tma(const CUtensorMap& src_map, T* dst, const Geometry& g,
                                       const StepConst<F2>& k, const AxisCoef<float>* tx,
                                       const AxisCoef<float>* ty, int variant, int grid,
                                       int* err, cudaStream_t st, int pdl, int polls) {
    if (polls < 0) polls = kTmaPolls;
    if (9 * g.plane >= (1ll << 32)) return cudaErrorInvalidValue;
    const int ntx = (g.nx + kTbW - 1) / kTbW, nty = (g.ny + kTbH - 1) / kTbH;
    const int ntiles = ntx * nty;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid < ntiles ? grid : ntiles);
    cfg.blockDim = dim3(TmaLaunch<T>::threads);
    cfg.dynamicSmemBytes = tma_smem_bytes<T>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const int pitch = static_cast<int>(g.pitch);
    const unsigned plane = static_cast<unsigned>(g.plane);
#define LBM_TMA_CASE(V)                                                                          \
    if (variant == V)                                                                            \
        return cudaLaunchKernelEx(&cfg, step_tb2_tma_kernel<T, V>, src_map, dst, g.nx, g.ny, pitch, \
                                  plane, k, tx, ty, ntx, ntiles, err, polls);
    LBM_TMA_CASE(kNone)
    LBM_TMA_CASE(kTypeI)
    LBM_TMA_CASE(kTypeII)
    LBM_TMA_CASE(kTypeIII)
    LBM_TMA_CASE(kViscous)
#undef LBM_TMA_CASE
    return cudaErrorInvalidValue;
}

// Raise every variant's dynamic shared-memory limit to the kernel's need (once
// per device, outside any stream capture) and report the CTAs one SM holds.
template <typename T>
inline cudaError_t prepare_step_tb2_tma(int* per_sm) {
    const int bytes = static_cast<int>(tma_smem_bytes<T>());
    cudaError_t e = cudaSuccess;
#define LBM_TMA_ATTR(V)                                                                     \
    if (e == cudaSuccess)                                                                   \
        e = cudaFuncSetAttribute(step_tb2_tma_kernel<T, V>,                                 \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    LBM_TMA_ATTR(kNone)
    LBM_TMA_ATTR(kTypeI)
    LBM_TMA_ATTR(kTypeII)
    LBM_TMA_ATTR(kTypeIII)
    LBM_TMA_ATTR(kViscous)
#undef LBM_TMA_ATTR
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_tb2_tma_kernel<T, kTypeII>,
                                                          TmaLaunch<T>::threads, tma_smem_bytes<T>());
    return e;
}

}  // namespace lbm
