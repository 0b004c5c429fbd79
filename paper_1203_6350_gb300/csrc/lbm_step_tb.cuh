// Two time steps per launch (temporal blocking) on the two-cells-per-thread
// arithmetic.  A block owns an output tile of kTbW x kTbH cells.
//
//  1. It pulls from HBM the post-collision state of time t around the tile
//     and collides the ring-extended region R1 (the tile plus one row above
//     and below and two columns on each side, to keep pairs aligned), giving
//     the post-collision state of time t + 1 on R1.  That state stays in
//     shared memory in FP32 whatever the storage format: for FP32 storage it
//     is exactly what a one-step kernel would store in HBM; for 16-bit
//     storage the intermediate time level is not rounded to 16 bits, so a
//     two-step launch rounds to the format once per two steps (and skips the
//     encode and decode of the intermediate level, ~12 of its ~150
//     instructions per cell and step).  Cells of R1 outside the lattice hold
//     the boundary value instead: zero deviation for the Dirichlet far field,
//     the wrapped cell for periodic.
//  2. After a block barrier it pulls time t + 1 from shared memory, collides
//     the tile and stores time t + 2 to HBM.
//
// Each launch moves 72 B per cell (FP32) for two steps instead of 144 B, at
// the price of colliding R1 (1.2x the tile) in the first half.
#pragma once

#include "lbm_step2.cuh"

namespace lbm {

constexpr int kTbW = 64;            // tile width (cells): 32 pairs
constexpr int kTbH = 16;            // tile height (rows)
constexpr int kTbThreads = 256;
constexpr int kR1W = kTbW + 4;      // R1: columns x0 - 2 .. x0 + kTbW + 1
constexpr int kR1H = kTbH + 2;      // R1: rows y0 - 1 .. y0 + kTbH
constexpr int kR1Pairs = kR1W / 2;  // pairs per R1 row
constexpr int kR1Plane = kR1W * kR1H;  // elements per plane in shared memory

// Whether the two-step tile chooses bulk or layer collision per warp (VOTE of
// collide_lanes).  FP32: yes, with the kernel held to three blocks per SM
// (80 registers): 2.6 % faster at 2048^2 with a 37-cell layer, level with a
// 128-cell one.  16-bit: per pair, which keeps the kernel at 64 registers and
// four blocks per SM; the vote measured 0.2-0.9 % slower there.
template <typename T>
constexpr bool kTbVote = sizeof(T) == 4;

// R1 in FP32 (44,064 bytes, inside the default 48 KB window) for every format.
template <typename T>
constexpr size_t tb_smem_bytes() {
    return 9 * kR1Plane * sizeof(float);
}

// Periodic image of coordinate c in [0, n).
__device__ __forceinline__ int wrap_coord(int c, int n) {
    c %= n;
    return c < 0 ? c + n : c;
}

// Pull the nine populations of the cells (ca, y) and (cb, y), both inside the
// lattice, with the boundary rule for their sources.
template <typename T, int BC>
__device__ __forceinline__ void pull_lanes(const T* __restrict__ s, unsigned plane, int pitch,
                                           int ca, int cb, int y, int nx, int ny, F2 (&v)[9]) {
    v[0] = f2(pull_one<T, BC, 0>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 0>(s, plane, pitch, cb, y, nx, ny));
    v[1] = f2(pull_one<T, BC, 1>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 1>(s, plane, pitch, cb, y, nx, ny));
    v[2] = f2(pull_one<T, BC, 2>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 2>(s, plane, pitch, cb, y, nx, ny));
    v[3] = f2(pull_one<T, BC, 3>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 3>(s, plane, pitch, cb, y, nx, ny));
    v[4] = f2(pull_one<T, BC, 4>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 4>(s, plane, pitch, cb, y, nx, ny));
    v[5] = f2(pull_one<T, BC, 5>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 5>(s, plane, pitch, cb, y, nx, ny));
    v[6] = f2(pull_one<T, BC, 6>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 6>(s, plane, pitch, cb, y, nx, ny));
    v[7] = f2(pull_one<T, BC, 7>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 7>(s, plane, pitch, cb, y, nx, ny));
    v[8] = f2(pull_one<T, BC, 8>(s, plane, pitch, ca, y, nx, ny),
              pull_one<T, BC, 8>(s, plane, pitch, cb, y, nx, ny));
}

// Two steps on the tile at (x0, y0) by a block of NT threads (any shape,
// numbered by thread_rank): src holds time t, dst receives time t + 2;
// sm is the block's tb_smem_bytes<T>() of shared memory (R1 in FP32).  Ends
// with a block barrier, so the caller may reuse sm for the next tile right away.
template <typename T, int VAR, int BC, int NT = kTbThreads>
__device__ __forceinline__ void tb2_tile(const T* __restrict__ src, T* __restrict__ dst, int nx,
                                         int ny, int pitch, unsigned plane, const StepConst<F2>& k,
                                         const AxisCoef<float>* __restrict__ tx,
                                         const AxisCoef<float>* __restrict__ ty, int x0, int y0,
                                         float* sm, int thread_rank) {
    // ---- step 1: time t (HBM) -> time t + 1 on R1 (shared memory) ----
    for (int p = thread_rank; p < kR1Pairs * kR1H; p += NT) {
        const int px = p % kR1Pairs, py = p / kR1Pairs;
        const int x = x0 - 2 + 2 * px, y = y0 - 1 + py;
        F2 v[9];
        bool keep_a = true, keep_b = true;  // Dirichlet: lanes outside hold the wall value 0
        if (x > 0 && x + 2 < nx && y > 0 && y + 1 < ny) {
            pull_pair_interior<T>(src, plane, static_cast<unsigned>(pitch),
                                  static_cast<unsigned>(y * pitch + x), v);
            collide_lanes<VAR, UnbiasedScale<T>::value, kTbVote<T>>(v, x, x + 1, y, k, tx, ty);
        } else {
            int ca = x, cb = x + 1, cy = y;
            if (BC == kPeriodic) {
                ca = wrap_coord(ca, nx);
                cb = wrap_coord(cb, nx);
                cy = wrap_coord(cy, ny);
            } else {
                const bool row_in = y >= 0 && y < ny;
                keep_a = row_in && ca >= 0 && ca < nx;
                keep_b = row_in && cb >= 0 && cb < nx;
                // lanes outside compute on a clamped cell; their result is dropped
                ca = min(max(ca, 0), nx - 1);
                cb = min(max(cb, 0), nx - 1);
                cy = min(max(cy, 0), ny - 1);
            }
            pull_lanes<T, BC>(src, plane, pitch, ca, cb, cy, nx, ny, v);
            collide_lanes<VAR, UnbiasedScale<T>::value, kTbVote<T>>(v, ca, cb, cy, k, tx, ty);
            if (!(keep_a && keep_b)) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    v[i] = f2(keep_a ? f2_lo(v[i]) : 0.0f, keep_b ? f2_hi(v[i]) : 0.0f);
            }
        }
        store_pair<float>(sm, kR1Plane, static_cast<unsigned>(py * kR1W + 2 * px), v);
    }
    __syncthreads();

    // ---- step 2: time t + 1 (shared memory) -> time t + 2 on the tile (HBM) ----
    for (int p = thread_rank; p < (kTbW / 2) * kTbH; p += NT) {
        const int qx = p % (kTbW / 2), qy = p / (kTbW / 2);
        const int x = x0 + 2 * qx, y = y0 + qy;
        if (x >= nx || y >= ny) continue;
        F2 v[9];
        pull_pair_interior<float, true>(sm, kR1Plane, kR1W,
                                        static_cast<unsigned>((qy + 1) * kR1W + 2 * qx + 2), v);
        collide_pair<VAR, UnbiasedScale<T>::value, kTbVote<T>>(v, x, y, nx, k, tx, ty);
        const unsigned o = static_cast<unsigned>(y * pitch + x);
        if (x + 1 < nx)
            store_pair<T>(dst, plane, o, v);
        else
            store_lo<T>(dst, plane, o, v);
    }
    __syncthreads();
}

// Blocks per SM the registers must allow: three with the vote (FP32); 0 leaves
// the choice to the compiler (64 registers for 16-bit storage, four blocks).
template <typename T, int VAR, int BC>
__global__ void __launch_bounds__(kTbThreads, kTbVote<T> ? 3 : 0)
    step_tb2_kernel(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny, int pitch,
                    unsigned plane, StepConst<F2> k, const AxisCoef<float>* __restrict__ tx,
                    const AxisCoef<float>* __restrict__ ty) {
    extern __shared__ __align__(16) unsigned char tb_raw[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    tb2_tile<T, VAR, BC>(src, dst, nx, ny, pitch, plane, k, tx, ty, blockIdx.x * kTbW,
                         blockIdx.y * kTbH, reinterpret_cast<float*>(tb_raw), threadIdx.x);
    asm volatile("griddepcontrol.launch_dependents;");
}

// Launch two steps (src holds time t, dst receives time t + 2); pdl as for
// the one-step kernels.  cudaErrorInvalidValue when the nine planes exceed
// 32-bit element offsets.
template <typename T>
cudaError_t launch_step_tb2_t(const void* src, void* dst, const Geometry& g,
                              const StepConst<F2>& k, const AxisCoef<float>* tx,
                              const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                              int pdl) {
    if (9 * g.plane >= (1ll << 32)) return cudaErrorInvalidValue;
    const T* s = static_cast<const T*>(src);
    T* d = static_cast<T*>(dst);
    const int pitch = static_cast<int>(g.pitch);
    const unsigned plane = static_cast<unsigned>(g.plane);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((g.nx + kTbW - 1) / kTbW, (g.ny + kTbH - 1) / kTbH);
    cfg.blockDim = dim3(kTbThreads);
    cfg.dynamicSmemBytes = tb_smem_bytes<T>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
#define LBM_TB2_CASE(V, B)                                                                       \
    if (variant == V && bc == B)                                                                 \
        return cudaLaunchKernelEx(&cfg, step_tb2_kernel<T, V, B>, s, d, g.nx, g.ny, pitch, plane, \
                                  k, tx, ty);
    LBM_TB2_CASE(kNone, kDirichlet)
    LBM_TB2_CASE(kTypeI, kDirichlet)
    LBM_TB2_CASE(kTypeII, kDirichlet)
    LBM_TB2_CASE(kTypeIII, kDirichlet)
    LBM_TB2_CASE(kViscous, kDirichlet)
    LBM_TB2_CASE(kNone, kPeriodic)
    LBM_TB2_CASE(kTypeI, kPeriodic)
    LBM_TB2_CASE(kTypeII, kPeriodic)
    LBM_TB2_CASE(kTypeIII, kPeriodic)
    LBM_TB2_CASE(kViscous, kPeriodic)
#undef LBM_TB2_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbm
