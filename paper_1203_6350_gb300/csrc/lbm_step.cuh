// Fused single-lattice step kernel: pull-stream, moments, rho*/j*, MRT
// relaxation, damping term, back-transform, store -- one pass over HBM per
// time step (9 loads + 9 stores per cell).
#pragma once

#include "d2q9_cell.cuh"

namespace lbm {

constexpr int kStepBX = 128;  // threads along x: four full warps on one row
constexpr int kStepBY = 2;    // rows per block

template <typename T, int VAR, int BC>
__global__ void __launch_bounds__(kStepBX* kStepBY)
    step_kernel(const T* __restrict__ src, T* __restrict__ dst, Geometry g,
                StepConst<typename Codec<T>::CT> k,
                const typename Codec<T>::CT* __restrict__ chi_x,
                const typename Codec<T>::CT* __restrict__ chi_y) {
    using CT = typename Codec<T>::CT;
    const int x = blockIdx.x * kStepBX + threadIdx.x;
    const int y = blockIdx.y * kStepBY + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const long long o = (long long)y * g.pitch + x;
    PullSites ps;
    ps.init<BC>(x, y, g);
    CT v[9];
    pull_all<T, BC>(src, g.plane, o, ps, v);
    CT chi = CT(0);
    if (VAR != kNone) chi = fmax(__ldg(chi_x + x), __ldg(chi_y + y));
    collide<CT, VAR>(v, chi, k);
    store_all<T>(dst, g.plane, o, v);
}

template <typename T>
cudaError_t launch_step_t(const void* src, void* dst, const Geometry& g,
                          const StepConst<typename Codec<T>::CT>& k,
                          const typename Codec<T>::CT* chi_x, const typename Codec<T>::CT* chi_y,
                          int variant, int bc, cudaStream_t st) {
    const dim3 block(kStepBX, kStepBY);
    const dim3 grid((g.nx + kStepBX - 1) / kStepBX, (g.ny + kStepBY - 1) / kStepBY);
    const T* s = static_cast<const T*>(src);
    T* d = static_cast<T*>(dst);
#define LBM_STEP_CASE(V, B)                                                        \
    if (variant == V && bc == B) {                                                 \
        step_kernel<T, V, B><<<grid, block, 0, st>>>(s, d, g, k, chi_x, chi_y);    \
        return cudaGetLastError();                                                 \
    }
    LBM_STEP_CASE(kNone, kDirichlet)
    LBM_STEP_CASE(kTypeI, kDirichlet)
    LBM_STEP_CASE(kTypeII, kDirichlet)
    LBM_STEP_CASE(kTypeIII, kDirichlet)
    LBM_STEP_CASE(kNone, kPeriodic)
    LBM_STEP_CASE(kTypeI, kPeriodic)
    LBM_STEP_CASE(kTypeII, kPeriodic)
    LBM_STEP_CASE(kTypeIII, kPeriodic)
#undef LBM_STEP_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbm
