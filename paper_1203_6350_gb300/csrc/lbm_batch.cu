// Batched time step: many independent lattices advanced together by
// persistent launches over a tile table, and the C ABI that manages the batch
// (lbm_batch_* in include/lbm.h).
//
// Each instance is a lattice of its own (size, rates, damping variant,
// boundary, reference state, absorbing profile) with its own double buffer.
// It is active for the global steps start <= s < end, so instances admitted
// at different times and with different step budgets share every launch and
// each takes exactly its own number of steps.  A launch advances one global
// step, or two (temporal blocking); an instance whose budget ends after the
// first of the two takes only that one.  Every launch swaps the buffers of
// the instances it advanced, so an instance's current buffer is the parity of
// the number of launches it took, which the host counts.
//
// The per-cell arithmetic is that of the single-lattice kernels (one cell per
// thread, the packed pair, the two-step tile), and it does not depend on the
// tile shape or on the other instances: within the batched path a lattice
// gives the same result, bit for bit, alone and in any mix.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_step_tma.cuh"

namespace lbm {

// Element type of the per-axis tables for a compute type (the packed pair
// reads the FP32 tables).
template <typename CT>
struct AxisOf {
    using type = CT;
};
template <>
struct AxisOf<F2> {
    using type = float;
};

// Device descriptor of one instance; CT is the compute type of its constants
// (double, float, or F2 for the two-cells-per-thread kernel).
template <typename CT>
struct BatchInst {
    void* buf[2];
    const AxisCoef<typename AxisOf<CT>::type>* tx;
    const AxisCoef<typename AxisOf<CT>::type>* ty;
    long long start, end;  // active for start <= step < end
    long long l0;          // global launch index of its first launch (buffer 0 holds time 0)
    long long plane;
    int nx, ny, pitch, variant, bc, pad;
    StepConst<CT> k;
};

struct BatchTile {
    int inst, x0, y0, pad;
};

// Blocks of 256 threads per SM the register allocation must allow (0 leaves
// it to the compiler): FP32 is fastest at 40 registers (6 blocks, a few bytes
// of spill) -- measured ahead of 48 and of the compiler's own 52 -- FP64 at 80
// (3 blocks); the 16-bit formats with the compiler's own choice.
template <typename T>
struct BatchMinBlocks {
    static constexpr int value = 0;
};
template <>
struct BatchMinBlocks<float> {
    static constexpr int value = 6;
};
template <>
struct BatchMinBlocks<double> {
    static constexpr int value = 3;
};

// Walk this block's tiles b, b + G, ... of the table, so that at any moment
// the G blocks sweep one compact stretch of it (a contiguous run per block
// spreads the DRAM accesses and measured 27 % slower).  The table lists each
// instance's tiles together: the block copies an instance descriptor to
// shared memory only when its next tile belongs to another instance.  It
// fetches the next tile entry, and the next tile's descriptor when that
// differs (one word per thread, held in a register), while it processes the
// current tile, so a switch costs two barriers and a shared-memory store.
// body(tile, descriptor, step, lpar) runs for the tiles of instances active
// at `step` (start <= step < end), the first global step of this launch
// (lpar = parity of the global launch index); every branch on the descriptor
// is block-uniform.  Blocks have at most 256 threads, as many as the largest
// descriptor has words.
template <typename Inst, typename Body>
__device__ __forceinline__ void walk_tiles(const Inst* __restrict__ insts,
                                           const BatchTile* __restrict__ tiles, int ntiles,
                                           long long step, int lpar, unsigned char* raw,
                                           Body& body) {
    const Inst& sd = *reinterpret_cast<const Inst*>(raw);
    constexpr int kWords = (int)(sizeof(Inst) / 4);
    static_assert(sizeof(Inst) % 4 == 0, "descriptor must be word-sized");
    static_assert(kWords <= 256, "one descriptor word per thread");
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int G = gridDim.x;
    int held = -1;      // instance whose descriptor is in shared memory
    int fetched = -1;   // instance whose descriptor word this thread holds in `word`
    unsigned word = 0;
    BatchTile next = (int)blockIdx.x < ntiles ? tiles[blockIdx.x] : BatchTile{};
    for (int t = blockIdx.x; t < ntiles; t += G) {
        const BatchTile tile = next;
        if (t + G < ntiles) next = tiles[t + G];
        if (tile.inst != held) {  // block-uniform
            if (fetched != tile.inst && tid < kWords)
                word = __ldg(reinterpret_cast<const unsigned*>(insts + tile.inst) + tid);
            __syncthreads();  // everyone is done with the previous descriptor
            if (tid < kWords) reinterpret_cast<unsigned*>(raw)[tid] = word;
            __syncthreads();
            held = tile.inst;
        }
        fetched = -1;
        if (t + G < ntiles && next.inst != tile.inst) {  // block-uniform
            if (tid < kWords)
                word = __ldg(reinterpret_cast<const unsigned*>(insts + next.inst) + tid);
            fetched = next.inst;
        }
        if (step < sd.start || step >= sd.end) continue;  // block-uniform
        body(tile, sd, step, lpar);
    }
}

// One cell per thread: the tile is tile_x x tile_y cells, blockDim =
// (tile_x, 256 / tile_x).
template <typename T>
struct CellTile {
    using CT = typename Codec<T>::CT;
    static constexpr bool UB = UnbiasedScale<T>::value;
    int tile_y;
    __device__ __forceinline__ void operator()(const BatchTile& tile, const BatchInst<CT>& sd,
                                               long long, int lpar) const {
        const int parity = lpar ^ (int)(sd.l0 & 1);
        const T* src = static_cast<const T*>(sd.buf[parity]);
        T* dst = static_cast<T*>(sd.buf[1 - parity]);
        const int plane = static_cast<int>(sd.plane);  // 9 * plane < 2^31 (checked on add)
        const int nx = sd.nx, ny = sd.ny, pitch = sd.pitch;
        const int x = tile.x0 + threadIdx.x;
        const bool interior = tile.x0 > 0 && tile.y0 > 0 && tile.x0 + (int)blockDim.x < nx &&
                              tile.y0 + tile_y < ny;
        for (int ry = threadIdx.y; ry < tile_y; ry += blockDim.y) {
            const int y = tile.y0 + ry;
            if (x >= nx || y >= ny) continue;
            const int o = y * pitch + x;
            CT v[9];
            PullSites ps;
            if (interior) {
                ps.interior(pitch);
                pull_all_b<T, kDirichlet, false>(src, plane, o, ps, v);
            } else if (sd.bc == kPeriodic) {
                ps.edge<kPeriodic>(x, y, nx, ny, pitch);
                pull_all_b<T, kPeriodic, true>(src, plane, o, ps, v);
            } else {
                ps.edge<kDirichlet>(x, y, nx, ny, pitch);
                pull_all_b<T, kDirichlet, true>(src, plane, o, ps, v);
            }
            switch (sd.variant) {
                case kTypeI: collide_cell<CT, kTypeI, UB>(v, x, y, sd.k, sd.tx, sd.ty); break;
                case kTypeII: collide_cell<CT, kTypeII, UB>(v, x, y, sd.k, sd.tx, sd.ty); break;
                case kTypeIII: collide_cell<CT, kTypeIII, UB>(v, x, y, sd.k, sd.tx, sd.ty); break;
                case kViscous: collide_cell<CT, kViscous, UB>(v, x, y, sd.k, sd.tx, sd.ty); break;
                default: collide_cell<CT, kNone, UB>(v, x, y, sd.k, sd.tx, sd.ty); break;
            }
            store_all_b<T>(dst, plane, o, v);
        }
    }
};

// Two cells per thread (packed FP32): the tile is tile_x x tile_y cells,
// blockDim = (tile_x / 2, 512 / tile_x); a thread steps the pair (x, x + 1)
// of each of its rows, with the single-lattice pair kernel's pull, collision
// and store.
template <typename T>
struct PairTile {
    static constexpr bool UB = UnbiasedScale<T>::value;
    int tile_y;
    __device__ __forceinline__ void operator()(const BatchTile& tile, const BatchInst<F2>& sd,
                                               long long, int lpar) const {
        const int parity = lpar ^ (int)(sd.l0 & 1);
        const T* src = static_cast<const T*>(sd.buf[parity]);
        T* dst = static_cast<T*>(sd.buf[1 - parity]);
        const unsigned plane = static_cast<unsigned>(sd.plane);  // 9 * plane < 2^31 (checked on add)
        const int nx = sd.nx, ny = sd.ny, pitch = sd.pitch;
        const int x = tile.x0 + 2 * threadIdx.x;
        if (x >= nx) return;
        for (int ry = threadIdx.y; ry < tile_y; ry += blockDim.y) {
            const int y = tile.y0 + ry;
            if (y >= ny) break;
            const unsigned o = static_cast<unsigned>(y * pitch + x);
            F2 v[9];
            if (x > 0 && x + 2 < nx && y > 0 && y + 1 < ny)
                pull_pair_interior<T>(src, plane, static_cast<unsigned>(pitch), o, v);
            else if (sd.bc == kPeriodic)
                pull_pair_edge<T, kPeriodic>(src, plane, pitch, x, y, nx, ny, v);
            else
                pull_pair_edge<T, kDirichlet>(src, plane, pitch, x, y, nx, ny, v);
            const auto& k = sd.k;  // the collisions choose bulk or layer per warp (VOTE)
            switch (sd.variant) {
                case kTypeI: collide_pair<kTypeI, UB, true>(v, x, y, nx, k, sd.tx, sd.ty); break;
                case kTypeII: collide_pair<kTypeII, UB, true>(v, x, y, nx, k, sd.tx, sd.ty); break;
                case kTypeIII:
                    collide_pair<kTypeIII, UB, true>(v, x, y, nx, k, sd.tx, sd.ty);
                    break;
                case kViscous:
                    collide_pair<kViscous, UB, true>(v, x, y, nx, k, sd.tx, sd.ty);
                    break;
                default: collide_pair<kNone, UB, true>(v, x, y, nx, k, sd.tx, sd.ty); break;
            }
            if (x + 1 < nx)
                store_pair<T>(dst, plane, o, v);
            else
                store_lo<T>(dst, plane, o, v);
        }
    }
};

// Classes of instances for the two-step kernel: damping variant x boundary.
// The tile table lists the tiles of each class together, and each class has
// a kernel of its own, so that a kernel holds one collision body (a kernel
// switching over all ten needed more registers than three blocks per SM
// allow and spilled).
constexpr int kClasses = 10;
__host__ __device__ constexpr int batch_class(int variant, int bc) {
    return (bc == kPeriodic ? 5 : 0) + variant;
}

// Two time steps per launch on 64 x 16 tiles through shared memory (the
// single-lattice two-step tile), for the instances active at both global
// steps; an instance whose budget ends after the first takes one step.
template <typename T, int VAR, int BC>
struct TwoStepTile {
    float* sm;  // R1 in FP32
    __device__ __forceinline__ void operator()(const BatchTile& tile, const BatchInst<F2>& sd,
                                               long long step, int lpar) const {
        const int parity = lpar ^ (int)(sd.l0 & 1);
        const T* src = static_cast<const T*>(sd.buf[parity]);
        T* dst = static_cast<T*>(sd.buf[1 - parity]);
        const unsigned plane = static_cast<unsigned>(sd.plane);
        const int nx = sd.nx, ny = sd.ny, pitch = sd.pitch;
        const int rank = threadIdx.x;
        if (step + 1 < sd.end) {  // block-uniform
            tb2_tile<T, VAR, BC>(src, dst, nx, ny, pitch, plane, sd.k, sd.tx, sd.ty, tile.x0,
                                 tile.y0, sm, rank);
            return;
        }
        // the last step of the budget: one step on the tile's pairs
        for (int p = rank; p < (kTbW / 2) * kTbH; p += kTbThreads) {
            const int x = tile.x0 + 2 * (p % (kTbW / 2)), y = tile.y0 + p / (kTbW / 2);
            if (x >= nx || y >= ny) continue;
            const unsigned o = static_cast<unsigned>(y * pitch + x);
            F2 v[9];
            if (x > 0 && x + 2 < nx && y > 0 && y + 1 < ny)
                pull_pair_interior<T>(src, plane, static_cast<unsigned>(pitch), o, v);
            else
                pull_pair_edge<T, BC>(src, plane, pitch, x, y, nx, ny, v);
            collide_pair<VAR, UnbiasedScale<T>::value>(v, x, y, nx, sd.k, sd.tx, sd.ty);
            if (x + 1 < nx)
                store_pair<T>(dst, plane, o, v);
            else
                store_lo<T>(dst, plane, o, v);
        }
    }
};

// The global step and launch counters of a batch, advanced on the device after
// each run of launches: counters[0] = step, counters[1] = launch.  A launch
// within a run reads counters + its offsets.

// One step of every active instance, one cell per thread.
template <typename T>
__global__ void __launch_bounds__(256, BatchMinBlocks<T>::value)
    batch_step_kernel(const BatchInst<typename Codec<T>::CT>* __restrict__ insts,
                      const BatchTile* __restrict__ tiles, const int* __restrict__ ntiles_p,
                      const long long* __restrict__ counters, int step_off, int launch_off,
                      int tile_y) {
    __shared__ __align__(16) unsigned char raw[sizeof(BatchInst<typename Codec<T>::CT>)];
    // the previous launch must have finished before any buffer is touched
    asm volatile("griddepcontrol.wait;" ::: "memory");
    CellTile<T> body{tile_y};
    walk_tiles(insts, tiles, *ntiles_p, counters[0] + step_off,
               (int)((counters[1] + launch_off) & 1), raw,
               body);
    asm volatile("griddepcontrol.launch_dependents;");
}

// One step of every active instance, two cells per thread.  At most 80
// registers (3 blocks per SM): left to itself the compiler keeps the packed
// descriptor constants in registers across the tile's rows and needs 116.
template <typename T>
__global__ void __launch_bounds__(256, 3)
    batch_step2_kernel(const BatchInst<F2>* __restrict__ insts, const BatchTile* __restrict__ tiles,
                       const int* __restrict__ ntiles_p, const long long* __restrict__ counters,
                       int step_off, int launch_off, int tile_y) {
    __shared__ __align__(16) unsigned char raw[sizeof(BatchInst<F2>)];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    PairTile<T> body{tile_y};
    walk_tiles(insts, tiles, *ntiles_p, counters[0] + step_off,
               (int)((counters[1] + launch_off) & 1), raw,
               body);
    asm volatile("griddepcontrol.launch_dependents;");
}

// Two steps of every active instance of class batch_class(VAR, BC) per launch
// (64 x 16 tiles, 256 threads, tb_smem_bytes<T>() of dynamic shared memory).
// table: [0] all tiles, [1 + 2c] first tile and [2 + 2c] tile count of class c.
template <typename T, int VAR, int BC>
__global__ void __launch_bounds__(kTbThreads, 3)
    batch_tb2_kernel(const BatchInst<F2>* __restrict__ insts, const BatchTile* __restrict__ tiles,
                     const int* __restrict__ table, const long long* __restrict__ counters,
                     int step_off, int launch_off) {
    __shared__ __align__(16) unsigned char raw[sizeof(BatchInst<F2>)];
    extern __shared__ __align__(16) unsigned char tb_raw[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    constexpr int c = batch_class(VAR, BC);
    TwoStepTile<T, VAR, BC> body{reinterpret_cast<float*>(tb_raw)};
    walk_tiles(insts, tiles + table[1 + 2 * c], table[2 + 2 * c], counters[0] + step_off,
               (int)((counters[1] + launch_off) & 1), raw, body);
    asm volatile("griddepcontrol.launch_dependents;");
}

// Two steps per launch on the Dirichlet instances of damping variant VAR,
// each tile's input staged by TMA as in step_tb2_tma_kernel: maps[2 i + p] is
// the tensor map of buffer p of dense instance i.  Thread 0 plans each tile
// from the instance's window -- skip (inactive), two staged steps, or the one
// step that ends a budget (pulled from global memory) -- and issues the next
// tile's copy as soon as step one has read the box.  Waits are bounded as in
// the single-lattice kernel; a CTA that gives up sets *err.
//
// A CTA's consecutive tiles are G apart in the table, so for small lattices
// nearly every tile belongs to another instance.  Nothing the next tile needs
// is fetched on the critical path: its tile record (one tile further ahead)
// and its instance descriptor arrive by cp.async into the other of two
// shared-memory slots while the current tile computes.
constexpr int kDescChunks = (int)(sizeof(BatchInst<F2>) / 8);  // 8-byte cp.async pieces
static_assert(sizeof(BatchInst<F2>) % 8 == 0 && kDescChunks <= kTmaThreads,
              "descriptor slots: 8-byte multiples, one 8-byte piece per thread");
constexpr size_t kTmaDescOff = kTmaBoxBytes + kTmaRingBytes + 16;  // box, ring, mbarrier, mode
static_assert(kTmaDescOff % 16 == 0, "16-byte aligned slots (the tile records follow)");

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int VAR>
__global__ void __launch_bounds__(kTmaThreads, 2)
    batch_tb2_tma_kernel(const BatchInst<F2>* __restrict__ insts,
                         const CUtensorMap* __restrict__ maps, const BatchTile* __restrict__ tiles,
                         const int* __restrict__ table, const long long* __restrict__ counters,
                         int step_off, int launch_off, int* __restrict__ err, int polls) {
    extern __shared__ __align__(128) unsigned char tma_raw[];
    float* box = reinterpret_cast<float*>(tma_raw);
    float* r1 = reinterpret_cast<float*>(tma_raw + kTmaBoxBytes);
    auto* bar = reinterpret_cast<unsigned long long*>(tma_raw + kTmaBoxBytes + kTmaRingBytes);
    auto* mode_sm = reinterpret_cast<int*>(tma_raw + kTmaBoxBytes + kTmaRingBytes + 8);
    // two descriptor slots, then two tile-record slots
    auto* desc = reinterpret_cast<BatchInst<F2>*>(tma_raw + kTmaDescOff);
    auto* trec = reinterpret_cast<BatchTile*>(tma_raw + kTmaDescOff + 2 * sizeof(BatchInst<F2>));
    constexpr int c = batch_class(VAR, kDirichlet);
    const int tid = threadIdx.x, G = gridDim.x;
    if (tid == 0) mbar_init(bar);
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const BatchTile* ct = tiles + table[1 + 2 * c];
    const int count = table[2 + 2 * c];
    const long long step = counters[0] + step_off;
    const int lpar = (int)((counters[1] + launch_off) & 1);
    // 0: inactive, 1: two staged steps (copy issued), 2: the budget's last step
    auto plan_and_issue = [&](const BatchTile& tl, const BatchInst<F2>& d) -> int {
        const long long st = d.start, en = d.end;
        if (step < st || step >= en) return 0;
        if (step + 1 >= en) return 2;
        const int parity = lpar ^ (int)(d.l0 & 1);
        tma_box_load(box, maps + 2 * tl.inst + parity, bar, tl.x0 - kTmaPad, tl.y0 - 2);
        return 1;
    };
    if ((int)blockIdx.x >= count) {
        asm volatile("griddepcontrol.launch_dependents;");
        return;
    }
    // the first tile's record and descriptor, and the second tile's record
    if (tid < 2) {
        const int t = blockIdx.x + tid * G;
        if (t < count) trec[tid] = ct[t];
    }
    __syncthreads();
    if (tid < kDescChunks)
        reinterpret_cast<unsigned long long*>(desc)[tid] =
            __ldg(reinterpret_cast<const unsigned long long*>(insts + trec[0].inst) + tid);
    __syncthreads();
    if (tid == 0) *mode_sm = plan_and_issue(trec[0], desc[0]);
    __syncthreads();
    unsigned phase = 0;
    int n = 0;
    for (int t = blockIdx.x; t < count; t += G, ++n) {
        const int sl = n & 1, so = sl ^ 1;
        const int mode = *mode_sm;  // block-uniform
        const BatchTile tile = trec[sl];
        const BatchInst<F2>& sd = desc[sl];
        const bool more = t + G < count;
        // the next tile's descriptor into the other slot, while this tile computes
        if (more && tid < kDescChunks)
            cp_async8(reinterpret_cast<unsigned long long*>(desc + so) + tid,
                      reinterpret_cast<const unsigned long long*>(insts + trec[so].inst) + tid);
        cp_async_commit();
        const int parity = lpar ^ (int)(sd.l0 & 1);
        const int nx = sd.nx, ny = sd.ny, pitch = sd.pitch;
        const unsigned plane = static_cast<unsigned>(sd.plane);
        float* dst = static_cast<float*>(sd.buf[1 - parity]);
        const int x0 = tile.x0, y0 = tile.y0;
        if (mode == 1) {
            const bool ok = mbar_wait(bar, phase, polls);
            phase ^= 1u;
            if (!__syncthreads_and(ok)) {  // the whole CTA stops together
                cp_async_wait_all();
                if (tid == 0) {
                    mbar_wait(bar, phase ^ 1u, kTmaDrainPolls);  // the copy in flight
                    atomicExch(err, 1);
                }
                return;
            }
            for (int p = tid; p < kR1Pairs * kR1H; p += kTmaThreads) {
                const int px = p % kR1Pairs, py = p / kR1Pairs;
                const int x = x0 - 2 + 2 * px, y = y0 - 1 + py;
                F2 v[9];
                pull_pair_interior<float, true>(
                    box, kTmaPlane, kTmaW,
                    static_cast<unsigned>((py + 1) * kTmaW + kTmaPad - 2 + 2 * px), v);
                const bool row_in = y >= 0 && y < ny;
                const bool keep_a = row_in && x >= 0 && x < nx;
                const bool keep_b = row_in && x + 1 >= 0 && x + 1 < nx;
                collide_lanes<VAR, true, true>(v, min(max(x, 0), nx - 1),
                                               min(max(x + 1, 0), nx - 1),
                                               min(max(y, 0), ny - 1), sd.k, sd.tx, sd.ty);
                if (!(keep_a && keep_b)) {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        v[i] = f2(keep_a ? f2_lo(v[i]) : 0.0f, keep_b ? f2_hi(v[i]) : 0.0f);
                }
                store_pair<float>(r1, kR1Plane, static_cast<unsigned>(py * kR1W + 2 * px), v);
            }
        }
        cp_async_wait_all();
        __syncthreads();  // the box is read; the next descriptor has arrived
        if (tid == 0) {
            *mode_sm = more ? plan_and_issue(trec[so], desc[so]) : 0;
            if (t + 2 * G < count) cp_async16(trec + sl, ct + (t + 2 * G));  // the record after
            cp_async_commit();
        }
        if (mode == 1) {
            for (int p = tid; p < (kTbW / 2) * kTbH; p += kTmaThreads) {
                const int qx = p % (kTbW / 2), qy = p / (kTbW / 2);
                const int x = x0 + 2 * qx, y = y0 + qy;
                if (x >= nx || y >= ny) continue;
                F2 v[9];
                pull_pair_interior<float, true>(
                    r1, kR1Plane, kR1W, static_cast<unsigned>((qy + 1) * kR1W + 2 * qx + 2), v);
                collide_pair<VAR, true, true>(v, x, y, nx, sd.k, sd.tx, sd.ty);
                const unsigned o = static_cast<unsigned>(y * pitch + x);
                if (x + 1 < nx)
                    store_pair<float, true>(dst, plane, o, v);
                else
                    store_lo<float>(dst, plane, o, v);
            }
        } else if (mode == 2) {  // the last step of the budget: one step from global memory
            const float* src = static_cast<const float*>(sd.buf[parity]);
            for (int p = tid; p < (kTbW / 2) * kTbH; p += kTmaThreads) {
                const int x = x0 + 2 * (p % (kTbW / 2)), y = y0 + p / (kTbW / 2);
                if (x >= nx || y >= ny) continue;
                const unsigned o = static_cast<unsigned>(y * pitch + x);
                F2 v[9];
                if (x > 0 && x + 2 < nx && y > 0 && y + 1 < ny)
                    pull_pair_interior<float>(src, plane, static_cast<unsigned>(pitch), o, v);
                else
                    pull_pair_edge<float, kDirichlet>(src, plane, pitch, x, y, nx, ny, v);
                collide_pair<VAR, true, true>(v, x, y, nx, sd.k, sd.tx, sd.ty);
                if (x + 1 < nx)
                    store_pair<float>(dst, plane, o, v);
                else
                    store_lo<float>(dst, plane, o, v);
            }
        }
        cp_async_wait_all();  // thread 0: the record after next has arrived
        __syncthreads();  // R1 and this slot's descriptor are read; *mode_sm is written
    }
    asm volatile("griddepcontrol.launch_dependents;");
}

constexpr size_t batch_tma_smem_bytes() {
    return kTmaDescOff + 2 * sizeof(BatchInst<F2>) + 2 * sizeof(BatchTile);
}

__global__ void advance_counters_kernel(long long* counters, int steps, int launches) {
    counters[0] += steps;
    counters[1] += launches;
}

// Kernel of a batch: cells per thread 1 or 2, steps per launch 1 or 2 (2
// needs cells == 2).
template <typename T>
const void* batch_kernel_ptr(int cells, int spl) {
    if (spl == 2) return reinterpret_cast<const void*>(&batch_tb2_kernel<T, kTypeII, kDirichlet>);
    if (cells == 2) return reinterpret_cast<const void*>(&batch_step2_kernel<T>);
    return reinterpret_cast<const void*>(&batch_step_kernel<T>);
}
template <>
const void* batch_kernel_ptr<double>(int, int) {
    return reinterpret_cast<const void*>(&batch_step_kernel<double>);
}

template <typename T>
size_t batch_smem(int spl) {
    return spl == 2 ? tb_smem_bytes<T>() : 0;
}

// The TMA-staged two-step kernel of Dirichlet class c (FP32 batches).
inline cudaError_t launch_tb2_tma_class(int c, cudaLaunchConfig_t cfg, const BatchInst<F2>* insts,
                                        const CUtensorMap* maps, const BatchTile* tiles,
                                        const int* table, const long long* counters, int step_off,
                                        int launch_off, int* err, int grid, int polls) {
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTmaThreads);
    cfg.dynamicSmemBytes = batch_tma_smem_bytes();
#define LBM_TB2_TMA_CLASS(V)                                                                  \
    if (c == batch_class(V, kDirichlet))                                                      \
        return cudaLaunchKernelEx(&cfg, batch_tb2_tma_kernel<V>, insts, maps, tiles, table,   \
                                  counters, step_off, launch_off, err, polls);
    LBM_TB2_TMA_CLASS(kNone)
    LBM_TB2_TMA_CLASS(kTypeI)
    LBM_TB2_TMA_CLASS(kTypeII)
    LBM_TB2_TMA_CLASS(kTypeIII)
    LBM_TB2_TMA_CLASS(kViscous)
#undef LBM_TB2_TMA_CLASS
    return cudaErrorInvalidValue;
}

// Shared-memory limits of the batched TMA kernels (outside any capture) and
// their CTAs per SM.
inline cudaError_t prepare_batch_tma(int* per_sm) {
    const int bytes = static_cast<int>(batch_tma_smem_bytes());
    cudaError_t e = cudaSuccess;
#define LBM_TB2_TMA_ATTR(V)                                                                 \
    if (e == cudaSuccess)                                                                   \
        e = cudaFuncSetAttribute(batch_tb2_tma_kernel<V>,                                   \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    LBM_TB2_TMA_ATTR(kNone)
    LBM_TB2_TMA_ATTR(kTypeI)
    LBM_TB2_TMA_ATTR(kTypeII)
    LBM_TB2_TMA_ATTR(kTypeIII)
    LBM_TB2_TMA_ATTR(kViscous)
#undef LBM_TB2_TMA_ATTR
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_tb2_tma_kernel<kTypeII>,
                                                          kTmaThreads, batch_tma_smem_bytes());
    return e;
}

// The two-step kernel of class c.
template <typename T>
cudaError_t launch_tb2_class(int c, cudaLaunchConfig_t& cfg, const BatchInst<F2>* insts,
                             const BatchTile* tiles, const int* table, const long long* counters,
                             int step_off, int launch_off) {
#define LBM_TB2_CLASS(V, B)                                                                    \
    if (c == batch_class(V, B))                                                                \
        return cudaLaunchKernelEx(&cfg, batch_tb2_kernel<T, V, B>, insts, tiles, table, counters, \
                                  step_off, launch_off);
    LBM_TB2_CLASS(kNone, kDirichlet)
    LBM_TB2_CLASS(kTypeI, kDirichlet)
    LBM_TB2_CLASS(kTypeII, kDirichlet)
    LBM_TB2_CLASS(kTypeIII, kDirichlet)
    LBM_TB2_CLASS(kViscous, kDirichlet)
    LBM_TB2_CLASS(kNone, kPeriodic)
    LBM_TB2_CLASS(kTypeI, kPeriodic)
    LBM_TB2_CLASS(kTypeII, kPeriodic)
    LBM_TB2_CLASS(kTypeIII, kPeriodic)
    LBM_TB2_CLASS(kViscous, kPeriodic)
#undef LBM_TB2_CLASS
    return cudaErrorInvalidValue;
}

// One batched launch: step_off / launch_off added to the device counters.
// Two-step launches run one kernel per class in class_mask, each a
// programmatic dependent of the one before.
// Staging of the two-step input by TMA in a batched launch: the Dirichlet
// classes of an FP32 batch use it when maps is set.
struct BatchTma {
    const CUtensorMap* maps = nullptr;
    int* err = nullptr;
    int grid = 0;
    int polls = kTmaPolls;  // each tile's wait for its staged copy
};

template <typename T>
cudaError_t launch_batch_t(const void* insts, const BatchTile* tiles, const int* ntiles,
                           const long long* counters, int step_off, int launch_off, int tile_x,
                           int tile_y, int grid, int cells, int spl, cudaStream_t st, int pdl,
                           int class_mask, const BatchTma& tma = BatchTma{}) {
    using CT = typename Codec<T>::CT;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = spl == 2 ? dim3(kTbThreads)
                 : cells == 2 ? dim3(tile_x / 2, 512 / tile_x) : dim3(tile_x, 256 / tile_x);
    cfg.dynamicSmemBytes = batch_smem<T>(spl);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const auto* ip2 = static_cast<const BatchInst<F2>*>(insts);
    if (spl == 2) {
        for (int c = 0; c < kClasses; ++c) {
            if (!((class_mask >> c) & 1)) continue;
            const bool staged = std::is_same<T, float>::value && tma.maps && c < 5;
            const cudaError_t e =
                staged ? launch_tb2_tma_class(c, cfg, ip2, tma.maps, tiles, ntiles, counters,
                                              step_off, launch_off, tma.err, tma.grid,
                                              tma.polls)
                       : launch_tb2_class<T>(c, cfg, ip2, tiles, ntiles, counters, step_off,
                                             launch_off);
            if (e != cudaSuccess) return e;
            cfg.numAttrs = 1;  // the next class depends on this one
        }
        return cudaSuccess;
    }
    if (cells == 2)
        return cudaLaunchKernelEx(&cfg, batch_step2_kernel<T>, ip2, tiles, ntiles, counters,
                                  step_off, launch_off, tile_y);
    return cudaLaunchKernelEx(&cfg, batch_step_kernel<T>, static_cast<const BatchInst<CT>*>(insts),
                              tiles, ntiles, counters, step_off, launch_off, tile_y);
}
template <>
cudaError_t launch_batch_t<double>(const void* insts, const BatchTile* tiles, const int* ntiles,
                                   const long long* counters, int step_off, int launch_off,
                                   int tile_x, int tile_y, int grid, int, int, cudaStream_t st,
                                   int pdl, int, const BatchTma&) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tile_x, 256 / tile_x);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, batch_step_kernel<double>,
                              static_cast<const BatchInst<double>*>(insts), tiles, ntiles, counters,
                              step_off, launch_off, tile_y);
}

}  // namespace lbm

using lbm::AxisCoef;
using lbm::BatchInst;
using lbm::BatchTile;
using lbm::Geometry;
using lbm::StepConst;

namespace {

constexpr int kBatchChunk = 32;  // steps per captured graph

struct Instance {
    int nx = 0, ny = 0;
    double rho0 = 1, ux0 = 0, uy0 = 0;
    double rho_f = 1, ux_f = 0, uy_f = 0;
    lbm_rates rates{};
    int variant = 0, bc = 0;
    int64_t budget = 0;
    int64_t start = INT64_MAX;  // global step at which it started (after init)
    int64_t l0 = 0;             // global launch index of its first launch
    int64_t launched = 0;       // launches that advanced it (its buffer is launched & 1)
    Geometry geo{};
    size_t buf_bytes = 0, tab_bytes = 0;
    void* buf[2] = {nullptr, nullptr};
    void* tabs = nullptr;  // AxisCoef x table followed by y table
    std::vector<unsigned char> tabs_host;  // the tables' host image (source of the upload)
    int bulk[4] = {0, 0, 0, 0};  // rectangle [x0, x1) x [y0, y1) where chi = 0
    bool initialised = false;
};

}  // namespace

struct lbm_batch_ctx {
    int storage = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    lbm_allocator alloc{};
    bool custom_alloc = false;
    std::map<int, Instance> insts;
    int next_id = 0;
    int64_t step = 0;      // global step (host mirror of d_counters[0])
    int64_t launches = 0;  // global launch index (host mirror of d_counters[1])
    int cpt = 1;           // cells per thread of the batched kernel (2 is the 16-bit default)
    int spl = 1;           // time steps per launch (2 needs cpt == 2)
    int tile_x = 128, tile_y = 8;
    int grid = 0;
    // device tables
    void* d_insts = nullptr;
    size_t insts_cap = 0;  // bytes
    BatchTile* d_tiles = nullptr;
    size_t tiles_cap = 0;  // entries
    int* d_ntiles = nullptr;  // [0] tiles, [1 + 2c] first tile and [2 + 2c] tiles of class c
    long long* d_counters = nullptr;  // [0] global step, [1] global launch
    double* d_diag = nullptr;
    double* staging = nullptr;
    size_t staging_bytes = 0;
    std::vector<int> dense;  // dense index -> instance id
    bool dirty = true;
    // host images of the device tables, kept as the source of their uploads
    std::vector<unsigned char> h_descs;
    std::vector<BatchTile> h_tiles;
    int h_ntiles[1 + 2 * lbm::kClasses] = {};  // host image of d_ntiles (256 bytes allocated)
    int class_mask = 0;  // classes with tiles
    int graph_mask = 0;  // classes the captured graph launches
    // TMA staging of the two-step input (FP32 batches, Dirichlet instances)
    bool tma = false;
    int tma_grid = 0;
    bool canary = false;  // LBM_CANARY=1 at creation: instances' row padding holds NaN canaries
    CUtensorMap* d_maps = nullptr;  // 2 per dense instance
    size_t maps_cap = 0;            // entries
    std::vector<CUtensorMap> h_maps;
    int* d_tma_err = nullptr;
    int tma_polls = lbm::kTmaPolls;  // each staged copy's wait (LBM_TMA_WAIT_POLLS overrides)
    // buffers of removed instances, freed once the launches issued before the
    // removal have completed (their event), so that removal never waits
    struct Retired {
        void* p;
        size_t bytes;
        cudaEvent_t ev;
    };
    std::vector<Retired> retired;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture_stream = nullptr;
    std::string err;
};

namespace {

int bfail(lbm_batch_ctx* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

void* bd_alloc(lbm_batch_ctx* b, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (b->custom_alloc) return b->alloc.alloc(bytes, b->alloc.ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void bd_free(lbm_batch_ctx* b, void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (b->custom_alloc)
        b->alloc.free(p, bytes, b->alloc.ctx);
    else
        cudaFree(p);
}

// Free the buffers of removed instances whose removal event has completed
// (all of them with wait = true, after the stream has drained).  Entries are
// grouped: an entry with an event is followed by the other buffers of the
// same instance (event nullptr).
void reap(lbm_batch_ctx* b, bool wait) {
    if (wait) cudaStreamSynchronize(b->stream);
    std::vector<lbm_batch_ctx::Retired> keep;
    bool done = true;
    for (auto& r : b->retired) {
        if (r.ev) {
            const cudaError_t q = cudaEventQuery(r.ev);
            done = wait || q == cudaSuccess;
            if (q != cudaSuccess && q != cudaErrorNotReady) cudaGetLastError();
            if (done) {
                cudaEventDestroy(r.ev);
                r.ev = nullptr;
                bd_free(b, r.p, r.bytes);
                continue;
            }
        } else if (done) {
            bd_free(b, r.p, r.bytes);
            continue;
        }
        keep.push_back(r);
    }
    b->retired.swap(keep);
}

struct BDeviceGuard {
    int prev = -1;
    explicit BDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~BDeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

size_t storage_size(int storage) { return lbm::storage_bytes(storage); }

Geometry geometry_of(int nx, int ny, int storage) {
    const size_t es = storage_size(storage);
    const long long per_row = (long long)((nx * es + 127) / 128 * 128 / es);
    return Geometry{nx, ny, per_row, per_row * ny};
}

template <typename CT>
StepConst<CT> consts_of(const Instance& in) {
    return lbm::make_step_const<CT>(in.rates.s, in.rates.n, in.rates.m, in.rho0, in.ux0, in.uy0,
                                    in.rho_f, in.ux_f, in.uy_f, in.bulk);
}

template <typename CT>
BatchInst<CT> desc_of(const Instance& in) {
    BatchInst<CT> d{};
    d.buf[0] = in.buf[0];
    d.buf[1] = in.buf[1];
    using A = AxisCoef<typename lbm::AxisOf<CT>::type>;
    d.tx = static_cast<const A*>(in.tabs);
    d.ty = static_cast<const A*>(in.tabs) + in.nx;
    d.start = in.initialised ? in.start : LLONG_MAX;
    d.end = in.initialised ? in.start + in.budget : LLONG_MAX;
    d.l0 = in.l0;
    d.plane = in.geo.plane;
    d.nx = in.nx;
    d.ny = in.ny;
    d.pitch = static_cast<int>(in.geo.pitch);
    d.variant = in.variant;
    d.bc = in.bc;
    d.k = consts_of<CT>(in);
    return d;
}

size_t desc_size(int storage, int cells) {
    if (storage == LBM_F64) return sizeof(BatchInst<double>);
    return cells == 2 ? sizeof(BatchInst<lbm::F2>) : sizeof(BatchInst<float>);
}

void drop_batch_graph(lbm_batch_ctx* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// One batched launch of `steps` (1 or 2) global steps; the offsets are added
// to the device counters (pending advances of this run of launches).
cudaError_t launch_batch(lbm_batch_ctx* b, cudaStream_t st, int steps, int step_off,
                         int launch_off, int pdl) {
    const int spl = steps == 2 ? 2 : 1;
    // in two-step mode the tile table holds two-step tiles; a one-step launch
    // covers them with the pair kernel
    const int tx = b->spl == 2 ? lbm::kTbW : b->tile_x;
    const int ty = b->spl == 2 ? lbm::kTbH : b->tile_y;
    switch (b->storage) {
        case LBM_F64:
            return lbm::launch_batch_t<double>(b->d_insts, b->d_tiles, b->d_ntiles, b->d_counters,
                                               step_off, launch_off, tx, ty, b->grid, 1, 1, st,
                                               pdl, b->class_mask);
        case LBM_F32:
            return lbm::launch_batch_t<float>(
                b->d_insts, b->d_tiles, b->d_ntiles, b->d_counters, step_off, launch_off, tx, ty,
                b->grid, b->cpt, spl, st, pdl, b->class_mask,
                lbm::BatchTma{b->tma ? b->d_maps : nullptr, b->d_tma_err, b->tma_grid,
                              b->tma_polls});
        case LBM_F16DEV:
            return lbm::launch_batch_t<__half>(b->d_insts, b->d_tiles, b->d_ntiles, b->d_counters,
                                               step_off, launch_off, tx, ty, b->grid, b->cpt, spl,
                                               st, pdl, b->class_mask);
        default:
            return lbm::launch_batch_t<__nv_bfloat16>(b->d_insts, b->d_tiles, b->d_ntiles,
                                                      b->d_counters, step_off, launch_off, tx, ty,
                                                      b->grid, b->cpt, spl, st, pdl,
                                                      b->class_mask);
    }
}

// Count, for every instance, the launches among `count` launches of `d` steps
// each, the first at global step step0, that advance it (those whose first
// step lies in its window [start, start + budget)).
void account(lbm_batch_ctx* b, int64_t step0, int d, int64_t count) {
    auto ceil_div = [](int64_t a, int64_t q) { return a >= 0 ? (a + q - 1) / q : -((-a) / q); };
    for (auto& kv : b->insts) {
        Instance& in = kv.second;
        if (!in.initialised) continue;
        const int64_t lo = std::max<int64_t>(0, ceil_div(in.start - step0, d));
        const int64_t hi = std::min<int64_t>(count, ceil_div(in.start + in.budget - step0, d));
        if (hi > lo) in.launched += hi - lo;
    }
}

cudaError_t compute_grid(lbm_batch_ctx* b) {
    const void* fn = nullptr;
    size_t smem = 0;
    switch (b->storage) {
        case LBM_F64: fn = lbm::batch_kernel_ptr<double>(1, 1); break;
        case LBM_F32:
            fn = lbm::batch_kernel_ptr<float>(b->cpt, b->spl);
            smem = lbm::batch_smem<float>(b->spl);
            break;
        case LBM_F16DEV:
            fn = lbm::batch_kernel_ptr<__half>(b->cpt, b->spl);
            smem = lbm::batch_smem<__half>(b->spl);
            break;
        default:
            fn = lbm::batch_kernel_ptr<__nv_bfloat16>(b->cpt, b->spl);
            smem = lbm::batch_smem<__nv_bfloat16>(b->spl);
            break;
    }
    int per_sm = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return e;
    b->grid = std::max(1, per_sm * sms);
    return cudaSuccess;
}

// Rebuild the descriptor array and the tile table on the device (stream-ordered).
int sync_tables(lbm_batch_ctx* b) {
    if (!b->dirty) return LBM_OK;
    b->dense.clear();
    std::vector<unsigned char>& descs = b->h_descs;
    std::vector<BatchTile>& tiles = b->h_tiles;
    descs.clear();
    tiles.clear();
    std::vector<BatchTile> per_class[lbm::kClasses];
    const size_t ds = desc_size(b->storage, b->cpt);
    for (auto& kv : b->insts) {
        const Instance& in = kv.second;
        const int di = static_cast<int>(b->dense.size());
        b->dense.push_back(kv.first);
        const size_t off = descs.size();
        descs.resize(off + ds);
        if (b->storage == LBM_F64) {
            const BatchInst<double> d = desc_of<double>(in);
            std::memcpy(descs.data() + off, &d, ds);
        } else if (b->cpt == 2) {
            const BatchInst<lbm::F2> d = desc_of<lbm::F2>(in);
            std::memcpy(descs.data() + off, &d, ds);
        } else {
            const BatchInst<float> d = desc_of<float>(in);
            std::memcpy(descs.data() + off, &d, ds);
        }
        if (!in.initialised) continue;
        const int tx = b->spl == 2 ? lbm::kTbW : b->tile_x;
        const int ty = b->spl == 2 ? lbm::kTbH : b->tile_y;
        std::vector<BatchTile>& out = per_class[lbm::batch_class(in.variant, in.bc)];
        for (int y0 = 0; y0 < in.ny; y0 += ty)
            for (int x0 = 0; x0 < in.nx; x0 += tx) out.push_back(BatchTile{di, x0, y0, 0});
    }
    // tensor maps of both buffers of every Dirichlet instance (FP32 two-step batches)
    if (b->tma && b->spl == 2) {
        b->h_maps.assign(2 * b->dense.size(), CUtensorMap{});
        for (size_t di = 0; di < b->dense.size(); ++di) {
            const Instance& in = b->insts.at(b->dense[di]);
            if (in.bc != LBM_BC_DIRICHLET_EQ) continue;
            for (int p = 0; p < 2; ++p)
                if (!lbm::encode_tma_map_f32(&b->h_maps[2 * di + p], in.buf[p], in.geo))
                    return bfail(b, LBM_ERR_CUDA, "the driver did not encode a tensor map");
        }
    }
    // the tiles of each class together (the two-step launch runs a kernel per class)
    int mask = 0;
    for (int c = 0; c < lbm::kClasses; ++c) {
        b->h_ntiles[1 + 2 * c] = static_cast<int>(tiles.size());
        b->h_ntiles[2 + 2 * c] = static_cast<int>(per_class[c].size());
        if (!per_class[c].empty()) mask |= 1 << c;
        tiles.insert(tiles.end(), per_class[c].begin(), per_class[c].end());
    }
    b->class_mask = mask;
    if (b->graph && b->spl == 2 && mask != b->graph_mask) drop_batch_graph(b);
    bool realloc = false;
    if (descs.size() > b->insts_cap) {
        cudaStreamSynchronize(b->stream);
        bd_free(b, b->d_insts, b->insts_cap);
        b->insts_cap = std::max(descs.size(), 2 * b->insts_cap);
        b->d_insts = bd_alloc(b, b->insts_cap);
        if (!b->d_insts) return bfail(b, LBM_ERR_OOM, "descriptor table allocation failed");
        realloc = true;
    }
    if (tiles.size() > b->tiles_cap) {
        cudaStreamSynchronize(b->stream);
        bd_free(b, b->d_tiles, b->tiles_cap * sizeof(BatchTile));
        b->tiles_cap = std::max(tiles.size(), 2 * b->tiles_cap);
        b->d_tiles = static_cast<BatchTile*>(bd_alloc(b, b->tiles_cap * sizeof(BatchTile)));
        if (!b->d_tiles) return bfail(b, LBM_ERR_OOM, "tile table allocation failed");
        realloc = true;
    }
    if (b->tma && b->spl == 2 && b->h_maps.size() > b->maps_cap) {
        cudaStreamSynchronize(b->stream);
        bd_free(b, b->d_maps, b->maps_cap * sizeof(CUtensorMap));
        b->maps_cap = std::max(b->h_maps.size(), 2 * b->maps_cap);
        b->d_maps = static_cast<CUtensorMap*>(bd_alloc(b, b->maps_cap * sizeof(CUtensorMap)));
        if (!b->d_maps) return bfail(b, LBM_ERR_OOM, "tensor map table allocation failed");
        realloc = true;
    }
    if (realloc) drop_batch_graph(b);
    cudaError_t e = cudaSuccess;
    if (b->tma && b->spl == 2 && !b->h_maps.empty())
        e = cudaMemcpyAsync(b->d_maps, b->h_maps.data(), b->h_maps.size() * sizeof(CUtensorMap),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !descs.empty())
        e = cudaMemcpyAsync(b->d_insts, descs.data(), descs.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !tiles.empty())
        e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile),
                            cudaMemcpyHostToDevice, b->stream);
    b->h_ntiles[0] = static_cast<int>(tiles.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_ntiles, b->h_ntiles, sizeof(b->h_ntiles), cudaMemcpyHostToDevice,
                            b->stream);
    // Stream-ordered after the launches that read the old tables.  The host
    // images live in the context, so nothing here waits for the device.
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch tables: ") + cudaGetErrorString(e));
    b->dirty = false;
    return LBM_OK;
}

cudaError_t ensure_batch_graph(lbm_batch_ctx* b) {
    if (b->graph) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!b->capture_stream) {
        e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const int n = kBatchChunk / b->spl;  // launches per chunk
    for (int k = 0; k < n && e == cudaSuccess; ++k)
        e = launch_batch(b, b->capture_stream, b->spl, k * b->spl, k, k > 0);
    if (e == cudaSuccess) {
        lbm::advance_counters_kernel<<<1, 1, 0, b->capture_stream>>>(b->d_counters, kBatchChunk, n);
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e == cudaSuccess) b->graph_mask = b->class_mask;
    return e;
}

// After the stream is synchronised: LBM_ERR_CUDA if a staged copy timed out.
int check_batch_tma(lbm_batch_ctx* b) {
    if (!b->d_tma_err) return LBM_OK;
    int flag = 0;
    const cudaError_t e = cudaMemcpy(&flag, b->d_tma_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("TMA error flag: ") + cudaGetErrorString(e));
    if (flag) return bfail(b, LBM_ERR_CUDA, "a TMA-staged copy did not complete within its wait");
    return LBM_OK;
}

Instance* find(lbm_batch_ctx* b, int id) {
    auto it = b->insts.find(id);
    return it == b->insts.end() ? nullptr : &it->second;
}

int64_t inst_time(const lbm_batch_ctx* b, const Instance& in) {
    if (!in.initialised) return 0;
    const int64_t t = b->step - in.start;
    return t < 0 ? 0 : (t > in.budget ? in.budget : t);
}

int ensure_bstaging(lbm_batch_ctx* b, size_t need) {
    if (b->staging && b->staging_bytes >= need) return LBM_OK;
    cudaStreamSynchronize(b->stream);
    bd_free(b, b->staging, b->staging_bytes);
    b->staging = static_cast<double*>(bd_alloc(b, need));
    b->staging_bytes = b->staging ? need : 0;
    if (!b->staging) return bfail(b, LBM_ERR_OOM, "staging allocation failed");
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_batch_instance_bytes(int nx, int ny, lbm_storage storage) {
    if (nx < 1 || ny < 1 || storage < LBM_F64 || storage > LBM_BF16DEV) return 0;
    const Geometry g = geometry_of(nx, ny, storage);
    const size_t cts = storage == LBM_F64 ? 8 : 4;
    return 2 * 9 * (size_t)g.plane * storage_size(storage) + 4 * cts * (size_t)(nx + ny);
}

int lbm_batch_create(lbm_storage storage, void* cuda_stream, const lbm_allocator* alloc,
                     lbm_batch* out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (storage < LBM_F64 || storage > LBM_BF16DEV) return LBM_ERR_ARG;
    if (alloc && (!alloc->alloc || !alloc->free)) return LBM_ERR_ARG;
    lbm_batch_ctx* b = new lbm_batch_ctx();
    b->storage = storage;
    b->canary = lbm::canary_requested();
    // 16-bit batches are issue-bound and gain from the packed pair (1.2x measured);
    // FP32 batches are memory-latency-bound and the one-cell kernel's higher
    // occupancy wins (1.04x).
    b->cpt = (storage == LBM_F16DEV || storage == LBM_BF16DEV) ? 2 : 1;
    if (const char* c = std::getenv("LBM_CPT")) {
        if (!std::strcmp(c, "1")) b->cpt = 1;
        if (!std::strcmp(c, "2") && storage != LBM_F64) b->cpt = 2;
    }
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (alloc) {
        b->alloc = *alloc;
        b->custom_alloc = true;
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = compute_grid(b);
    if (e != cudaSuccess) {
        delete b;
        return LBM_ERR_CUDA;
    }
    static_assert(sizeof(b->h_ntiles) <= 256, "tile counts must fit their allocation");
    b->d_ntiles = static_cast<int*>(bd_alloc(b, 256));
    b->d_counters = static_cast<long long*>(bd_alloc(b, 256));
    b->d_diag = static_cast<double*>(bd_alloc(b, sizeof(double) * (lbm::kDiagBlocks * lbm::kDiag + lbm::kDiag)));
    if (!b->d_ntiles || !b->d_counters || !b->d_diag) {
        lbm_batch_destroy(b);
        return LBM_ERR_OOM;
    }
    e = cudaMemsetAsync(b->d_ntiles, 0, sizeof(b->h_ntiles), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(long long), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return LBM_ERR_CUDA;
    }
    if (const char* t = std::getenv("LBM_BATCH_TILE")) {
        int tx = 0, ty = 0;
        if (std::sscanf(t, "%dx%d", &tx, &ty) == 2) lbm_batch_set_tiling(b, tx, ty);
    }
    // FP32 batches stage the two-step input of their Dirichlet instances by TMA
    // (LBM_BATCH_TMA=0 keeps plain loads)
    const char* tma_env = std::getenv("LBM_BATCH_TMA");
    if (storage == LBM_F32 && !(tma_env && !std::strcmp(tma_env, "0"))) {
        int per_sm = 0, sms = 0;
        e = lbm::prepare_batch_tma(&per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        b->d_tma_err = static_cast<int*>(bd_alloc(b, 256));
        if (e == cudaSuccess && per_sm > 0 && b->d_tma_err &&
            cudaMemsetAsync(b->d_tma_err, 0, sizeof(int), b->stream) == cudaSuccess &&
            cudaStreamSynchronize(b->stream) == cudaSuccess) {
            b->tma = true;
            b->tma_grid = per_sm * sms;
            const int polls = lbm::tma_wait_polls();
            if (polls >= 0) b->tma_polls = polls;
        }
        cudaGetLastError();
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch b, int tile_x, int tile_y) {
    if (!b) return LBM_ERR_ARG;
    if (!(tile_x == 32 || tile_x == 64 || tile_x == 128 || tile_x == 256))
        return bfail(b, LBM_ERR_ARG, "tile_x must be 32, 64, 128 or 256");
    if (tile_y < 1 || tile_y > 256 || (tile_y % (256 / tile_x)) != 0)
        return bfail(b, LBM_ERR_ARG, "tile_y must be a multiple of 256 / tile_x, at most 256");
    b->tile_x = tile_x;
    b->tile_y = tile_y;
    b->dirty = true;
    drop_batch_graph(b);
    return LBM_OK;
}

int lbm_batch_set_cells_per_thread(lbm_batch b, int cells) {
    if (!b) return LBM_ERR_ARG;
    if (cells != 1 && cells != 2) return bfail(b, LBM_ERR_ARG, "cells per thread must be 1 or 2");
    if (cells == 2 && b->storage == LBM_F64)
        return bfail(b, LBM_ERR_ARG, "two cells per thread needs FP32 or 16-bit storage");
    if (cells == b->cpt) return LBM_OK;
    BDeviceGuard dg(b->device);
    cudaStreamSynchronize(b->stream);
    drop_batch_graph(b);  // the captured launches name the other kernel
    b->cpt = cells;
    if (cells == 1) b->spl = 1;
    b->dirty = true;      // the descriptors change type
    const cudaError_t e = compute_grid(b);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("grid: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_batch_cells_per_thread(lbm_batch b) { return b ? b->cpt : LBM_ERR_ARG; }

int lbm_batch_set_steps_per_launch(lbm_batch b, int steps) {
    if (!b) return LBM_ERR_ARG;
    if (steps != 1 && steps != 2) return bfail(b, LBM_ERR_ARG, "steps per launch must be 1 or 2");
    if (steps == 2 && b->cpt != 2)
        return bfail(b, LBM_ERR_ARG, "two steps per launch needs two cells per thread");
    if (steps == b->spl) return LBM_OK;
    BDeviceGuard dg(b->device);
    cudaStreamSynchronize(b->stream);
    drop_batch_graph(b);  // the captured launches name the other kernel
    b->spl = steps;
    b->dirty = true;      // the tile table changes shape
    const cudaError_t e = compute_grid(b);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("grid: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_batch_steps_per_launch(lbm_batch b) { return b ? b->spl : LBM_ERR_ARG; }

int lbm_batch_tma_staging(lbm_batch b) { return b ? (b->tma ? 1 : 0) : LBM_ERR_ARG; }

int lbm_batch_add(lbm_batch b, int nx, int ny, double rho0, double ux0, double uy0,
                  const lbm_rates* rates, lbm_bc bc, lbm_variant variant, const double* chi_x,
                  const double* chi_y, double rho_ref, double ux_ref, double uy_ref, int64_t nsteps,
                  int* id) {
    if (!b) return LBM_ERR_ARG;
    if (!id || !rates || !chi_x || !chi_y) return bfail(b, LBM_ERR_ARG, "NULL argument");
    if (nx < 1 || ny < 1 || nsteps < 0) return bfail(b, LBM_ERR_ARG, "bad size or step budget");
    if (bc != LBM_BC_DIRICHLET_EQ && bc != LBM_BC_PERIODIC) return bfail(b, LBM_ERR_ARG, "bad bc");
    if (variant < LBM_SPONGE_NONE || variant > LBM_SPONGE_VISCOUS) return bfail(b, LBM_ERR_ARG, "bad variant");
    if (variant == LBM_SPONGE_VISCOUS && chi_x && chi_y) {
        for (int i = 0; i < nx; ++i)
            if (chi_x[i] > 1.0) return bfail(b, LBM_ERR_ARG, "viscous sponge: layer fraction above 1");
        for (int i = 0; i < ny; ++i)
            if (chi_y[i] > 1.0) return bfail(b, LBM_ERR_ARG, "viscous sponge: layer fraction above 1");
    }
    if (!(rho0 > 0) || !(rho_ref > 0) || !std::isfinite(ux0) || !std::isfinite(uy0) ||
        !std::isfinite(ux_ref) || !std::isfinite(uy_ref))
        return bfail(b, LBM_ERR_ARG, "bad far-field or reference state");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(rates->s[i])) return bfail(b, LBM_ERR_ARG, "non-finite rate");
    if (!std::isfinite(rates->n) || !std::isfinite(rates->m) || rates->n < 0 || rates->m < 0)
        return bfail(b, LBM_ERR_ARG, "bad Guo weights");
    for (int i = 0; i < nx; ++i)
        if (!(chi_x[i] >= 0) || !std::isfinite(chi_x[i])) return bfail(b, LBM_ERR_ARG, "bad chi_x");
    for (int i = 0; i < ny; ++i)
        if (!(chi_y[i] >= 0) || !std::isfinite(chi_y[i])) return bfail(b, LBM_ERR_ARG, "bad chi_y");
    Instance in;
    in.nx = nx;
    in.ny = ny;
    in.rho0 = rho0;
    in.ux0 = ux0;
    in.uy0 = uy0;
    in.rho_f = rho_ref;
    in.ux_f = ux_ref;
    in.uy_f = uy_ref;
    in.rates = *rates;
    in.variant = variant;
    in.bc = bc;
    in.budget = nsteps;
    lbm::zero_run(chi_x, nx, in.bulk[0], in.bulk[1]);
    lbm::zero_run(chi_y, ny, in.bulk[2], in.bulk[3]);
    in.geo = geometry_of(nx, ny, b->storage);
    if (9 * in.geo.plane > 2147483647LL)
        return bfail(b, LBM_ERR_ARG, "lattice too large for the batched path (9 planes must hold "
                                     "fewer than 2^31 elements)");
    in.buf_bytes = 9 * (size_t)in.geo.plane * storage_size(b->storage);
    const size_t cts = b->storage == LBM_F64 ? 8 : 4;
    in.tab_bytes = 4 * cts * (size_t)(nx + ny);
    BDeviceGuard dg(b->device);
    in.buf[0] = bd_alloc(b, in.buf_bytes);
    in.buf[1] = bd_alloc(b, in.buf_bytes);
    in.tabs = bd_alloc(b, in.tab_bytes);
    if (!in.buf[0] || !in.buf[1] || !in.tabs) {
        bd_free(b, in.buf[0], in.buf_bytes);
        bd_free(b, in.buf[1], in.buf_bytes);
        bd_free(b, in.tabs, in.tab_bytes);
        return bfail(b, LBM_ERR_OOM, "instance allocation failed");
    }
    const double nn = rates->n, mm = rates->m;
    cudaError_t e;
    // The host image stays with the instance, so the upload needs no wait.
    in.tabs_host.assign(in.tab_bytes, 0);
    if (b->storage == LBM_F64) {
        double* t = reinterpret_cast<double*>(in.tabs_host.data());
        for (int i = 0; i < nx + ny; ++i) {
            const double c = i < nx ? chi_x[i] : chi_y[i - nx];
            t[4 * i] = c;
            t[4 * i + 1] = 1.0 / (1.0 + nn * c);
            t[4 * i + 2] = 1.0 / (1.0 + mm * c);
            t[4 * i + 3] = 0.0;
        }
    } else {
        float* t = reinterpret_cast<float*>(in.tabs_host.data());
        for (int i = 0; i < nx + ny; ++i) {
            const double c = i < nx ? chi_x[i] : chi_y[i - nx];
            t[4 * i] = (float)c;
            t[4 * i + 1] = (float)(1.0 / (1.0 + nn * c));
            t[4 * i + 2] = (float)(1.0 / (1.0 + mm * c));
            t[4 * i + 3] = 0.0f;
        }
    }
    e = cudaMemcpyAsync(in.tabs, in.tabs_host.data(), in.tab_bytes, cudaMemcpyHostToDevice, b->stream);
    for (int i = 0; i < 2 && e == cudaSuccess && b->canary; ++i)
        e = lbm::paint_canary(in.buf[i], storage_size(b->storage), nx, in.geo.pitch, 9ll * ny,
                              b->stream);
    if (e != cudaSuccess) {
        bd_free(b, in.buf[0], in.buf_bytes);
        bd_free(b, in.buf[1], in.buf_bytes);
        bd_free(b, in.tabs, in.tab_bytes);
        return bfail(b, LBM_ERR_CUDA, std::string("lbm_batch_add: ") + cudaGetErrorString(e));
    }
    const int nid = b->next_id++;
    b->insts[nid] = in;
    b->dirty = true;
    *id = nid;
    return LBM_OK;
}

int lbm_batch_init_equilibrium(lbm_batch b, int id, const double* rho, const double* ux,
                               const double* uy, int on_device) {
    if (!b) return LBM_ERR_ARG;
    Instance* in = find(b, id);
    if (!in) return bfail(b, LBM_ERR_ARG, "unknown instance");
    if (!rho || !ux || !uy) return bfail(b, LBM_ERR_ARG, "field pointer is NULL");
    BDeviceGuard dg(b->device);
    const double *dr = rho, *dx = ux, *dy = uy;
    cudaError_t e = cudaSuccess;
    const size_t n = (size_t)in->nx * in->ny;
    if (!on_device) {
        int rc = ensure_bstaging(b, 3 * n * sizeof(double));
        if (rc) return rc;
        e = cudaMemcpyAsync(b->staging, rho, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->staging + n, ux, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->staging + 2 * n, uy, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        dr = b->staging;
        dx = b->staging + n;
        dy = b->staging + 2 * n;
    }
    if (e == cudaSuccess)
        e = lbm::launch_init(b->storage, in->buf[0], in->geo, lbm::BaseState{in->rho0, in->ux0, in->uy0},
                             dr, dx, dy, in->bc, b->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("lbm_batch_init_equilibrium: ") + cudaGetErrorString(e));
    in->initialised = true;
    in->start = b->step;
    in->l0 = b->launches;
    in->launched = 0;
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_init_pulse(lbm_batch b, int id, double eps, double half_width, double x0,
                         double y0) {
    if (!b) return LBM_ERR_ARG;
    Instance* in = find(b, id);
    if (!in) return bfail(b, LBM_ERR_ARG, "unknown instance");
    if (!std::isfinite(eps) || !(half_width > 0) || !std::isfinite(half_width) ||
        !std::isfinite(x0) || !std::isfinite(y0))
        return bfail(b, LBM_ERR_ARG, "pulse parameters must be finite with half_width > 0");
    BDeviceGuard dg(b->device);
    const cudaError_t e = lbm::launch_init_pulse(b->storage, in->buf[0], in->geo,
                                                 lbm::BaseState{in->rho0, in->ux0, in->uy0}, eps,
                                                 half_width, x0, y0, in->bc, b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("lbm_batch_init_pulse: ") + cudaGetErrorString(e));
    in->initialised = true;
    in->start = b->step;
    in->l0 = b->launches;
    in->launched = 0;
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int nsteps) {
    const lbm::NvtxRange nvtx("lbm_batch_step");
    if (!b) return LBM_ERR_ARG;
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps < 0");
    BDeviceGuard dg(b->device);
    int rc = sync_tables(b);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(b->stream, &cs);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "cudaStreamIsCapturing");
    if (cs == cudaStreamCaptureStatusNone && nsteps >= kBatchChunk) {
        e = ensure_batch_graph(b);
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        const int n = kBatchChunk / b->spl;
        while (nsteps >= kBatchChunk) {
            e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
            account(b, b->step, b->spl, n);
            b->step += kBatchChunk;
            b->launches += n;
            nsteps -= kBatchChunk;
        }
    }
    int step_off = 0, launch_off = 0;
    while (nsteps > 0) {
        const int d = (b->spl == 2 && nsteps >= 2) ? 2 : 1;
        e = launch_batch(b, b->stream, d, step_off, launch_off, launch_off > 0);
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
        account(b, b->step + step_off, d, 1);
        step_off += d;
        ++launch_off;
        nsteps -= d;
    }
    if (launch_off > 0) {
        lbm::advance_counters_kernel<<<1, 1, 0, b->stream>>>(b->d_counters, step_off, launch_off);
        e = cudaGetLastError();
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch advance: ") + cudaGetErrorString(e));
        b->step += step_off;
        b->launches += launch_off;
    }
    return LBM_OK;
}

int64_t lbm_batch_time(lbm_batch b, int id) {
    if (!b) return -1;
    Instance* in = find(b, id);
    return in ? inst_time(b, *in) : -1;
}

int lbm_batch_moments(lbm_batch b, int id, double* rho_dev, double* ux, double* uy, int on_device) {
    if (!b) return LBM_ERR_ARG;
    Instance* in = find(b, id);
    if (!in) return bfail(b, LBM_ERR_ARG, "unknown instance");
    if (!in->initialised) return bfail(b, LBM_ERR_STATE, "instance not initialised");
    BDeviceGuard dg(b->device);
    const size_t n = (size_t)in->nx * in->ny;
    double *dr = rho_dev, *dx = ux, *dy = uy;
    if (!on_device) {
        int rc = ensure_bstaging(b, 3 * n * sizeof(double));
        if (rc) return rc;
        dr = rho_dev ? b->staging : nullptr;
        dx = ux ? b->staging + n : nullptr;
        dy = uy ? b->staging + 2 * n : nullptr;
    }
    const int cur = (int)(in->launched & 1);
    cudaError_t e = lbm::launch_moments(b->storage, in->buf[cur], in->geo,
                                        lbm::BaseState{in->rho0, in->ux0, in->uy0}, in->bc, dr, dx, dy,
                                        b->stream, lbm::LineSource{});
    if (e == cudaSuccess && !on_device) {
        if (rho_dev) e = cudaMemcpyAsync(rho_dev, dr, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess && ux) e = cudaMemcpyAsync(ux, dx, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess && uy) e = cudaMemcpyAsync(uy, dy, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("lbm_batch_moments: ") + cudaGetErrorString(e));
    return on_device ? LBM_OK : check_batch_tma(b);
}

size_t lbm_batch_state_bytes(lbm_batch b, int id) {
    const Instance* in = b ? find(b, id) : nullptr;
    return in ? in->buf_bytes : 0;
}

int lbm_batch_get_state(lbm_batch b, int id, void* dst, size_t bytes, int on_device) {
    if (!b) return LBM_ERR_ARG;
    Instance* in = find(b, id);
    if (!in) return bfail(b, LBM_ERR_ARG, "unknown instance");
    if (!in->initialised) return bfail(b, LBM_ERR_STATE, "instance not initialised");
    if (!dst || bytes != in->buf_bytes)
        return bfail(b, LBM_ERR_ARG, "dst / bytes do not match lbm_batch_state_bytes");
    BDeviceGuard dg(b->device);
    const int cur = (int)(in->launched & 1);
    cudaError_t e = cudaMemcpyAsync(dst, in->buf[cur], bytes,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    b->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bfail(b, LBM_ERR_CUDA, std::string("lbm_batch_get_state: ") + cudaGetErrorString(e));
    return on_device ? LBM_OK : check_batch_tma(b);
}

int lbm_batch_diagnostics(lbm_batch b, int id, int x0, int y0, int x1, int y1, double out[6]) {
    if (!b) return LBM_ERR_ARG;
    Instance* in = find(b, id);
    if (!in || !out) return bfail(b, LBM_ERR_ARG, "unknown instance or NULL out");
    if (!in->initialised) return bfail(b, LBM_ERR_STATE, "instance not initialised");
    if (x0 < 0 || y0 < 0 || x1 > in->nx || y1 > in->ny || x0 > x1 || y0 > y1)
        return bfail(b, LBM_ERR_ARG, "region outside the lattice");
    BDeviceGuard dg(b->device);
    const int cur = (int)(in->launched & 1);
    double* res = b->d_diag + lbm::kDiagBlocks * lbm::kDiag;
    cudaError_t e = lbm::launch_diagnostics(b->storage, in->buf[cur], in->geo,
                                            lbm::BaseState{in->rho0, in->ux0, in->uy0}, in->bc, x0,
                                            y0, x1, y1, b->d_diag, res, b->stream, lbm::LineSource{});
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, lbm::kDiag * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("lbm_batch_diagnostics: ") + cudaGetErrorString(e));
    if (const int rc = check_batch_tma(b)) return rc;
    if (out[5] > 0) return bfail(b, LBM_ERR_NONFINITE, "the instance holds non-finite values");
    return LBM_OK;
}

int lbm_batch_remove(lbm_batch b, int id) {
    if (!b) return LBM_ERR_ARG;
    Instance* in = find(b, id);
    if (!in) return bfail(b, LBM_ERR_ARG, "unknown instance");
    BDeviceGuard dg(b->device);
    // launches already issued may still read its buffers: free them once an
    // event recorded now has completed (checked here and on later calls)
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, b->stream);
    if (e != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
        cudaStreamSynchronize(b->stream);  // fall back to waiting
    }
    b->retired.push_back({in->buf[0], in->buf_bytes, ev});
    b->retired.push_back({in->buf[1], in->buf_bytes, nullptr});
    b->retired.push_back({in->tabs, in->tab_bytes, nullptr});
    b->insts.erase(id);
    b->dirty = true;
    reap(b, false);
    return LBM_OK;
}

int lbm_batch_count(lbm_batch b) { return b ? static_cast<int>(b->insts.size()) : -1; }

int lbm_batch_set_stream(lbm_batch b, void* cuda_stream) {
    if (!b) return LBM_ERR_ARG;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    return LBM_OK;
}

const char* lbm_batch_last_error(lbm_batch b) { return b ? b->err.c_str() : ""; }

void lbm_batch_destroy(lbm_batch b) {
    if (!b) return;
    BDeviceGuard dg(b->device);
    cudaStreamSynchronize(b->stream);
    reap(b, true);
    drop_batch_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (auto& kv : b->insts) {
        bd_free(b, kv.second.buf[0], kv.second.buf_bytes);
        bd_free(b, kv.second.buf[1], kv.second.buf_bytes);
        bd_free(b, kv.second.tabs, kv.second.tab_bytes);
    }
    bd_free(b, b->d_insts, b->insts_cap);
    bd_free(b, b->d_tiles, b->tiles_cap * sizeof(BatchTile));
    bd_free(b, b->d_ntiles, 256);
    bd_free(b, b->d_maps, b->maps_cap * sizeof(CUtensorMap));
    bd_free(b, b->d_tma_err, 256);
    bd_free(b, b->d_counters, 256);
    bd_free(b, b->d_diag, sizeof(double) * (lbm::kDiagBlocks * lbm::kDiag + lbm::kDiag));
    bd_free(b, b->staging, b->staging_bytes);
    delete b;
}

}  // extern "C"
