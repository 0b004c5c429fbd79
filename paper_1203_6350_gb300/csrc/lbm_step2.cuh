// Two-cells-per-thread step kernel.  Each thread steps the neighbouring cells
// (x, x + 1), x even, of one row: the whole collision runs on packed FP32
// pairs (one add/sub/mul/fma .f32x2 instruction per operation for both
// cells), the three planes that do not move along x (i = 0, 2, 4) are pulled
// with one 64-bit (FP32) or 32-bit (16-bit storage) load per pair, and all
// nine planes are stored with one such access per pair.  The six planes that
// move along x are pulled cell by cell (two 32- or 16-bit loads; a pair of
// sources straddles the pair boundary).  Same scheme, same layout, same
// boundary rules as the one-cell kernel.
#pragma once

#include "lbm_step.cuh"

namespace lbm {

// Blocks of 128 threads (128 cells x 2 rows): measured 5 % faster than 256-thread
// blocks on the L2-resident 1024^2 lattice (finer-grained blocks leave less of
// the last wave idle), equal on HBM-bound lattices.
constexpr int kPairBX = 64;  // threads along x: 128 cells, two full warps
constexpr int kPairBY = 2;   // rows per block

// Storage of a pair of cells <-> F2.  Raw2 is the raw word of two adjacent
// elements (lo = cell x).
template <typename T>
struct PairCodec;
template <>
struct PairCodec<float> {
    using Raw2 = unsigned long long;
    template <int I>
    __device__ static __forceinline__ F2 dec2(Raw2 w) { return F2{w}; }
    template <int I>
    __device__ static __forceinline__ F2 dec11(float a, float b) { return f2(a, b); }
    template <int I>
    __device__ static __forceinline__ Raw2 enc2(F2 v) { return v.u; }
    template <int I>
    __device__ static __forceinline__ float enc_lo(F2 v) { return f2_lo(v); }
};

// 16-bit formats, FP16 as q_i = g_i 2^e_i (see scale_exp), BF16 as g_i.  FP16
// decodes each element with one mixed-precision FMA, q_i * 2^-e_i + (-0) in
// FP32: exact, the sign of a zero kept; it encodes by scaling the pair in FP32
// and converting both cells in one instruction.  BF16 converts both ways with
// no scale.
template <typename H, typename H2>
struct PairCodec16 {
    using Raw2 = unsigned;
    static constexpr bool kScaled = std::is_same<H, __half>::value;
    template <int I>
    __device__ static __forceinline__ F2 dec2(Raw2 w) {
        H2 h;
        memcpy(&h, &w, sizeof w);
        return dec11<I>(h.x, h.y);
    }
    template <int I>
    __device__ static __forceinline__ F2 dec11(H a, H b) {
        if constexpr (kScaled)
            return f2(dec_scaled<I>(a), dec_scaled<I>(b));
        else
            return f2(to_f(a), to_f(b));
    }
    template <int I>
    __device__ static __forceinline__ Raw2 enc2(F2 v) {
        if constexpr (kScaled) v = mul(v, lit<F2>(pow2f(scale_exp(I))));
        const H2 h = pack(f2_lo(v), f2_hi(v));
        Raw2 w;
        memcpy(&w, &h, sizeof w);
        return w;
    }
    template <int I>
    __device__ static __forceinline__ H enc_lo(F2 v) {
        return Codec<H>::template enc<I>(f2_lo(v));
    }
    // FP16 q times 2^-scale_exp(I) (a normal FP16 power of two) in FP32.
    template <int I>
    __device__ static __forceinline__ float dec_scaled(__half q) {
        static_assert(scale_exp(I) <= 14, "2^-e must be a normal FP16 number");
        const unsigned short s = static_cast<unsigned short>((15 - scale_exp(I)) << 10);
        float r;
        asm("fma.rn.f32.f16 %0, %1, %2, %3;"
            : "=f"(r)
            : "h"(__half_as_ushort(q)), "h"(s), "f"(-0.0f));
        return r;
    }
    __device__ static __forceinline__ float to_f(__half h) { return __half2float(h); }
    __device__ static __forceinline__ float to_f(__nv_bfloat16 h) { return __bfloat162float(h); }
    __device__ static __forceinline__ __half2 pack_h(float lo, float hi, __half2*) {
        return __floats2half2_rn(lo, hi);
    }
    __device__ static __forceinline__ __nv_bfloat162 pack_h(float lo, float hi, __nv_bfloat162*) {
        return __floats2bfloat162_rn(lo, hi);
    }
    __device__ static __forceinline__ H2 pack(float lo, float hi) {
        return pack_h(lo, hi, static_cast<H2*>(nullptr));
    }
};
template <>
struct PairCodec<__half> : PairCodec16<__half, __half2> {};
template <>
struct PairCodec<__nv_bfloat16> : PairCodec16<__nv_bfloat16, __nv_bfloat162> {};

// Loads of one element or one pair: through the read-only data path from
// global memory (SHARED = false) or plain loads from shared memory.
template <typename T, bool SHARED>
__device__ __forceinline__ T ld_one(const T* p) {
    if (SHARED) return *p;
    return __ldg(p);
}
template <typename T, bool SHARED>
__device__ __forceinline__ typename PairCodec<T>::Raw2 ld_pair(const T* p) {
    const auto* q = reinterpret_cast<const typename PairCodec<T>::Raw2*>(p);
    if (SHARED) return *q;
    return __ldg(q);
}

// Pull the nine populations of the pair at element offset o (row y, x even)
// of a store of 9 planes (`plane` elements apart) of rows `pitch` elements
// long, all sources inside the store.  Element offsets are 32-bit unsigned:
// valid while the nine planes hold fewer than 2^32 elements.
template <typename T, bool SHARED = false>
__device__ __forceinline__ void pull_pair_interior(const T* __restrict__ s, unsigned plane,
                                                   unsigned pitch, unsigned o, F2 (&v)[9]) {
    using PC = PairCodec<T>;
    const unsigned up = o - pitch, dn = o + pitch;  // rows y - 1, y + 1
    v[0] = PC::template dec2<0>(ld_pair<T, SHARED>(s + o));
    v[2] = PC::template dec2<2>(ld_pair<T, SHARED>(s + (2 * plane + up)));  // from (x, y - 1)
    v[4] = PC::template dec2<4>(ld_pair<T, SHARED>(s + (4 * plane + dn)));  // from (x, y + 1)
    const T* p1 = s + (plane + o);                                           // from (x - 1, y)
    v[1] = PC::template dec11<1>(ld_one<T, SHARED>(p1 - 1), ld_one<T, SHARED>(p1));
    const T* p3 = s + (3 * plane + o);                                       // from (x + 1, y)
    v[3] = PC::template dec11<3>(ld_one<T, SHARED>(p3 + 1), ld_one<T, SHARED>(p3 + 2));
    const T* p5 = s + (5 * plane + up);                                      // from (x - 1, y - 1)
    v[5] = PC::template dec11<5>(ld_one<T, SHARED>(p5 - 1), ld_one<T, SHARED>(p5));
    const T* p6 = s + (6 * plane + up);                                      // from (x + 1, y - 1)
    v[6] = PC::template dec11<6>(ld_one<T, SHARED>(p6 + 1), ld_one<T, SHARED>(p6 + 2));
    const T* p7 = s + (7 * plane + dn);                                      // from (x + 1, y + 1)
    v[7] = PC::template dec11<7>(ld_one<T, SHARED>(p7 + 1), ld_one<T, SHARED>(p7 + 2));
    const T* p8 = s + (8 * plane + dn);                                      // from (x - 1, y + 1)
    v[8] = PC::template dec11<8>(ld_one<T, SHARED>(p8 - 1), ld_one<T, SHARED>(p8));
}

// Population I of cell (c, y) pulled from (c - c_ix, y - c_iy) with the
// boundary rule: a Dirichlet far-field wall contributes a zero deviation,
// periodic wraps, the channel wraps y, takes the source population src_pop[I] at
// its left edge and the last column's own value at its right edge (outflow).
// The phantom cell c = nx of an odd-width lattice reads nothing (its result
// is never stored).
template <typename T, int BC, int I>
__device__ __forceinline__ float pull_one(const T* __restrict__ s, unsigned plane, int pitch,
                                          int c, int y, int nx, int ny,
                                          const float* src_pop = nullptr) {
    if (c >= nx) return 0.0f;
    int sx = c - cx(I), sy = y - cy(I);
    if (BC == kPeriodic) {
        sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
    } else if (BC == kChannel) {
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        if (sx < 0) return src_pop[I];
        if (sx >= nx) sx = nx - 1;
    } else if (sx < 0 || sx >= nx || sy < 0 || sy >= ny) {
        return 0.0f;
    }
    return Codec<T>::template dec<I>(__ldg(s + (I * plane + static_cast<unsigned>(sy * pitch + sx))));
}

template <typename T, int BC, int I>
__device__ __forceinline__ F2 pull_pair_one(const T* __restrict__ s, unsigned plane, int pitch,
                                            int x, int y, int nx, int ny, const float* src_pop) {
    return f2(pull_one<T, BC, I>(s, plane, pitch, x, y, nx, ny, src_pop),
              pull_one<T, BC, I>(s, plane, pitch, x + 1, y, nx, ny, src_pop));
}

template <typename T, int BC>
__device__ __forceinline__ void pull_pair_edge(const T* __restrict__ s, unsigned plane, int pitch,
                                               int x, int y, int nx, int ny, F2 (&v)[9],
                                               const float* src_pop = nullptr) {
    v[0] = pull_pair_one<T, BC, 0>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[1] = pull_pair_one<T, BC, 1>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[2] = pull_pair_one<T, BC, 2>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[3] = pull_pair_one<T, BC, 3>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[4] = pull_pair_one<T, BC, 4>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[5] = pull_pair_one<T, BC, 5>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[6] = pull_pair_one<T, BC, 6>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[7] = pull_pair_one<T, BC, 7>(s, plane, pitch, x, y, nx, ny, src_pop);
    v[8] = pull_pair_one<T, BC, 8>(s, plane, pitch, x, y, nx, ny, src_pop);
}

// STREAM stores with the evict-first policy (st.global.cs): for a lattice far
// larger than L2, whose output is not read again before L2 has turned over,
// so that it does not push out input lines a neighbouring tile still needs.
template <typename T, int I, bool STREAM = false>
__device__ __forceinline__ void store_pair_plane(T* __restrict__ d, unsigned plane, unsigned o,
                                                 const F2 (&v)[9]) {
    auto* p = reinterpret_cast<typename PairCodec<T>::Raw2*>(d + (I * plane + o));
    const typename PairCodec<T>::Raw2 w = PairCodec<T>::template enc2<I>(v[I]);
    if constexpr (STREAM)
        __stcs(p, w);
    else
        *p = w;
}

template <typename T, bool STREAM = false>
__device__ __forceinline__ void store_pair(T* __restrict__ d, unsigned plane, unsigned o,
                                           const F2 (&v)[9]) {
    store_pair_plane<T, 0, STREAM>(d, plane, o, v);
    store_pair_plane<T, 1, STREAM>(d, plane, o, v);
    store_pair_plane<T, 2, STREAM>(d, plane, o, v);
    store_pair_plane<T, 3, STREAM>(d, plane, o, v);
    store_pair_plane<T, 4, STREAM>(d, plane, o, v);
    store_pair_plane<T, 5, STREAM>(d, plane, o, v);
    store_pair_plane<T, 6, STREAM>(d, plane, o, v);
    store_pair_plane<T, 7, STREAM>(d, plane, o, v);
    store_pair_plane<T, 8, STREAM>(d, plane, o, v);
}

// Store only cell x of the pair (the last column of an odd-width lattice).
template <typename T>
__device__ __forceinline__ void store_lo(T* __restrict__ d, unsigned plane, unsigned o,
                                         const F2 (&v)[9]) {
    d[o] = PairCodec<T>::template enc_lo<0>(v[0]);
    d[plane + o] = PairCodec<T>::template enc_lo<1>(v[1]);
    d[2 * plane + o] = PairCodec<T>::template enc_lo<2>(v[2]);
    d[3 * plane + o] = PairCodec<T>::template enc_lo<3>(v[3]);
    d[4 * plane + o] = PairCodec<T>::template enc_lo<4>(v[4]);
    d[5 * plane + o] = PairCodec<T>::template enc_lo<5>(v[5]);
    d[6 * plane + o] = PairCodec<T>::template enc_lo<6>(v[6]);
    d[7 * plane + o] = PairCodec<T>::template enc_lo<7>(v[7]);
    d[8 * plane + o] = PairCodec<T>::template enc_lo<8>(v[8]);
}

// Collide a pair of cells of row y at columns xa (lo lane) and xb (hi lane),
// both inside the lattice.  Both cells take the damping path as soon as one
// of them lies in the layer; with chi = 0 that path is the plain relaxation
// bit for bit (rho* = rho, j* = j, no damping term, the bulk's tables holding
// chi = 0 and Guo factors 1; collide_layer and collide_viscous are written so
// that the arithmetic coincides), so where the choice is made changes no
// result.
//
// VOTE makes that choice for all the lanes that arrive together (a warp vote)
// instead of lane by lane: a warp across the edge of the bulk would otherwise
// run both paths one after the other.  Measured where layer edges do not fall
// on warp boundaries: the TMA-staged batched kernel 9.5 % faster on 256 mixed
// lattices, the one-step pair kernel and the single-lattice TMA kernel 5 %
// faster with a 37-cell layer (1024^2, 4096^2), no change with aligned edges.
// In the plain-load two-step kernel the vote raises the register count (FP16:
// 64 to 98, FP32: 77 to 90, 16-25 % slower as compiled freely); with FP32 held
// to three blocks per SM it gains, for 16-bit storage that kernel decides pair
// by pair (kTbVote).
template <int VAR, bool UB = true, bool VOTE = false>
__device__ __forceinline__ void collide_lanes(F2 (&v)[9], int xa, int xb, int y,
                                              const StepConst<F2>& k,
                                              const AxisCoef<float>* __restrict__ tx,
                                              const AxisCoef<float>* __restrict__ ty) {
    const unsigned lanes = VOTE ? __activemask() : 0u;
    const bool bulk = xa >= k.bulk_x0 && xa < k.bulk_x1 && xb >= k.bulk_x0 && xb < k.bulk_x1 &&
                      y >= k.bulk_y0 && y < k.bulk_y1;
    if (VAR == kNone || (VOTE ? __all_sync(lanes, bulk) : bulk)) {
        collide_bulk<F2, UB>(v, k);
        return;
    }
    const AxisCoef<float> a0 = load_coef(tx, xa), a1 = load_coef(tx, xb);
    const AxisCoef<float> ay = load_coef(ty, y);
    const float c0 = fmaxf(a0.chi, ay.chi), c1 = fmaxf(a1.chi, ay.chi);
    const bool layer = c0 > 0.0f || c1 > 0.0f;
    if (VOTE ? __any_sync(lanes, layer) : layer) {
        if (VAR == kViscous)  // the tables' chi slot holds the layer fraction r
            collide_viscous<F2, UB>(v, f2(c0, c1), k);
        else
            collide_layer<F2, VAR, UB>(v, f2(c0, c1),
                                       f2(fminf(a0.rn, ay.rn), fminf(a1.rn, ay.rn)),
                                       f2(fminf(a0.rm, ay.rm), fminf(a1.rm, ay.rm)), k);
    } else {
        collide_bulk<F2, UB>(v, k);
    }
}

// The pair (x, x + 1) of row y; the phantom cell x + 1 = nx of an odd-width
// lattice borrows the coefficients of its neighbour (its result is dropped).
template <int VAR, bool UB = true, bool VOTE = false>
__device__ __forceinline__ void collide_pair(F2 (&v)[9], int x, int y, int nx,
                                             const StepConst<F2>& k,
                                             const AxisCoef<float>* __restrict__ tx,
                                             const AxisCoef<float>* __restrict__ ty) {
    collide_lanes<VAR, UB, VOTE>(v, x, min(x + 1, nx - 1), y, k, tx, ty);
}

template <typename T, int VAR, int BC>
__global__ void __launch_bounds__(kPairBX* kPairBY)
    step2_kernel(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny, int pitch,
                 unsigned plane, StepConst<F2> k, const AxisCoef<float>* __restrict__ tx,
                 const AxisCoef<float>* __restrict__ ty, LineSource ls) {
    const int x = 2 * (blockIdx.x * kPairBX + threadIdx.x);
    const int y = blockIdx.y * kPairBY + threadIdx.y;
    // Launched as a programmatic dependent of the previous step: wait until that
    // grid has completed and its stores are visible.  No-op otherwise.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (x >= nx || y >= ny) {
        asm volatile("griddepcontrol.launch_dependents;");
        return;
    }
    const unsigned o = static_cast<unsigned>(y * pitch + x);
    // per thread: both cells and all their sources inside the lattice
    const bool interior = x > 0 && x + 2 < nx && y > 0 && y + 1 < ny;
    F2 v[9];
    if (interior) {
        pull_pair_interior<T>(src, plane, static_cast<unsigned>(pitch), o, v);
    } else {
        // the channel's source edge: its deviation scale at this step
        const float* src_pop = (BC == kChannel && x == 0) ? ls.pop + 9 * ls.t_off : nullptr;
        pull_pair_edge<T, BC>(src, plane, pitch, x, y, nx, ny, v, src_pop);
    }
    collide_pair<VAR, UnbiasedScale<T>::value, true>(v, x, y, nx, k, tx, ty);
    if (x + 1 < nx)
        store_pair<T>(dst, plane, o, v);
    else
        store_lo<T>(dst, plane, o, v);
    asm volatile("griddepcontrol.launch_dependents;");
}

// Launch one step of the pair kernel (storage float, __half or
// __nv_bfloat16); pdl as for the one-cell kernel.  Returns
// cudaErrorInvalidValue when the nine planes exceed 32-bit element offsets.
template <typename T>
cudaError_t launch_step2_t(const void* src, void* dst, const Geometry& g, const StepConst<F2>& k,
                           const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                           int bc, cudaStream_t st, int pdl, const LineSource& ls) {
    if (9 * g.plane >= (1ll << 32)) return cudaErrorInvalidValue;
    const T* s = static_cast<const T*>(src);
    T* d = static_cast<T*>(dst);
    const int pitch = static_cast<int>(g.pitch);
    const unsigned plane = static_cast<unsigned>(g.plane);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((g.nx + 2 * kPairBX - 1) / (2 * kPairBX), (g.ny + kPairBY - 1) / kPairBY);
    cfg.blockDim = dim3(kPairBX, kPairBY);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
#define LBM_STEP2_CASE(V, B)                                                                  \
    if (variant == V && bc == B)                                                              \
        return cudaLaunchKernelEx(&cfg, step2_kernel<T, V, B>, s, d, g.nx, g.ny, pitch, plane, k, \
                                  tx, ty, ls);
    LBM_STEP2_CASE(kNone, kDirichlet)
    LBM_STEP2_CASE(kTypeI, kDirichlet)
    LBM_STEP2_CASE(kTypeII, kDirichlet)
    LBM_STEP2_CASE(kTypeIII, kDirichlet)
    LBM_STEP2_CASE(kViscous, kDirichlet)
    LBM_STEP2_CASE(kNone, kPeriodic)
    LBM_STEP2_CASE(kTypeI, kPeriodic)
    LBM_STEP2_CASE(kTypeII, kPeriodic)
    LBM_STEP2_CASE(kTypeIII, kPeriodic)
    LBM_STEP2_CASE(kViscous, kPeriodic)
    LBM_STEP2_CASE(kNone, kChannel)
    LBM_STEP2_CASE(kTypeI, kChannel)
    LBM_STEP2_CASE(kTypeII, kChannel)
    LBM_STEP2_CASE(kTypeIII, kChannel)
    LBM_STEP2_CASE(kViscous, kChannel)
#undef LBM_STEP2_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbm
