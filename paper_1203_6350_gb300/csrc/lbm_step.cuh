// Fused single-lattice step kernel: pull-stream, moments, rho*/j*, MRT
// relaxation, damping term, back-transform, store -- one pass over HBM per
// time step (9 loads + 9 stores per cell).
#pragma once

#include "d2q9_cell.cuh"

namespace lbm {

constexpr int kStepBX = 128;  // threads along x: four full warps on one row
constexpr int kStepBY = 2;    // rows per block

template <typename CT>
__device__ __forceinline__ AxisCoef<CT> load_coef(const AxisCoef<CT>* t, int i);
template <>
__device__ __forceinline__ AxisCoef<float> load_coef(const AxisCoef<float>* t, int i) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(t) + i);
    return AxisCoef<float>{v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ AxisCoef<double> load_coef(const AxisCoef<double>* t, int i) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(t) + 2 * i);
    const double2 b = __ldg(reinterpret_cast<const double2*>(t) + 2 * i + 1);
    return AxisCoef<double>{a.x, a.y, b.x, b.y};
}

// Collide the pulled populations of one cell in place.
template <typename CT, int VAR, bool UB = true>
__device__ __forceinline__ void collide_cell(CT (&v)[9], int x, int y, const StepConst<CT>& k,
                                             const AxisCoef<CT>* tx, const AxisCoef<CT>* ty) {
    if (VAR == kNone || (x >= k.bulk_x0 && x < k.bulk_x1 && y >= k.bulk_y0 && y < k.bulk_y1)) {
        collide_bulk<CT, UB>(v, k);  // no layer here: skip the per-axis tables
    } else if (VAR == kViscous) {  // the tables' chi slot holds the layer fraction r
        const CT r = fmax(load_coef(tx, x).chi, load_coef(ty, y).chi);
        if (r > CT(0))
            collide_viscous<CT, UB>(v, r, k);
        else
            collide_bulk<CT, UB>(v, k);
    } else {
        const AxisCoef<CT> ax = load_coef(tx, x), ay = load_coef(ty, y);
        const CT chi = fmax(ax.chi, ay.chi);
        if (chi > CT(0))
            collide_layer<CT, VAR, UB>(v, chi, fmin(ax.rn, ay.rn), fmin(ax.rm, ay.rm), k);
        else
            collide_bulk<CT, UB>(v, k);
    }
}

template <typename T, int VAR, int BC>
__global__ void __launch_bounds__(kStepBX* kStepBY)
    step_kernel(PlanePtrs<T> src, PlanePtrs<T> dst, int nx, int ny, int pitch,
                StepConst<typename Codec<T>::CT> k,
                const AxisCoef<typename Codec<T>::CT>* __restrict__ tx,
                const AxisCoef<typename Codec<T>::CT>* __restrict__ ty, LineSource ls) {
    using CT = typename Codec<T>::CT;
    const int bx0 = blockIdx.x * kStepBX, by0 = blockIdx.y * kStepBY;
    const int x = bx0 + threadIdx.x;
    const int y = by0 + threadIdx.y;
    // block-uniform: every cell of the tile has all eight neighbours inside
    const bool interior = bx0 > 0 && by0 > 0 && bx0 + kStepBX < nx && by0 + kStepBY < ny;
    // Launched as a programmatic dependent of the previous step: wait until that
    // grid has completed and its stores are visible before touching either
    // buffer (it read the buffer this step writes).  No-op otherwise.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (x >= nx || y >= ny) {
        asm volatile("griddepcontrol.launch_dependents;");
        return;
    }
    const int o = y * pitch + x;
    CT v[9];
    PullSites ps;
    if (interior) {
        ps.interior(pitch);
        pull_all<T, BC, false>(src, o, ps, v);
    } else {
        ps.edge<BC>(x, y, nx, ny, pitch);
        // the channel's source edge: its deviation scale at this step
        const double src_s = (BC == kChannel && x == 0) ? line_source_scale(ls) : 0.0;
        pull_all<T, BC, true>(src, o, ps, v, src_s, ls.e);
    }
    collide_cell<CT, VAR, UnbiasedScale<T>::value>(v, x, y, k, tx, ty);
    store_all<T>(dst, o, v);
    // let the next step's grid launch while this one drains
    asm volatile("griddepcontrol.launch_dependents;");
}

// Launch one step; pdl != 0 launches it as a programmatic dependent of the
// previous kernel in the stream (its prologue overlaps that kernel's tail).
template <typename T>
cudaError_t launch_step_t(const void* src, void* dst, const Geometry& g,
                          const StepConst<typename Codec<T>::CT>& k,
                          const AxisCoef<typename Codec<T>::CT>* tx,
                          const AxisCoef<typename Codec<T>::CT>* ty, int variant, int bc,
                          cudaStream_t st, int pdl, const LineSource& ls) {
    const PlanePtrs<T> s = plane_ptrs<T>(const_cast<void*>(src), g.plane);
    const PlanePtrs<T> d = plane_ptrs<T>(dst, g.plane);
    const int pitch = static_cast<int>(g.pitch);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((g.nx + kStepBX - 1) / kStepBX, (g.ny + kStepBY - 1) / kStepBY);
    cfg.blockDim = dim3(kStepBX, kStepBY);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
#define LBM_STEP_CASE(V, B)                                                                  \
    if (variant == V && bc == B)                                                             \
        return cudaLaunchKernelEx(&cfg, step_kernel<T, V, B>, s, d, g.nx, g.ny, pitch, k, tx, ty, ls);
    LBM_STEP_CASE(kNone, kDirichlet)
    LBM_STEP_CASE(kTypeI, kDirichlet)
    LBM_STEP_CASE(kTypeII, kDirichlet)
    LBM_STEP_CASE(kTypeIII, kDirichlet)
    LBM_STEP_CASE(kViscous, kDirichlet)
    LBM_STEP_CASE(kNone, kPeriodic)
    LBM_STEP_CASE(kTypeI, kPeriodic)
    LBM_STEP_CASE(kTypeII, kPeriodic)
    LBM_STEP_CASE(kTypeIII, kPeriodic)
    LBM_STEP_CASE(kViscous, kPeriodic)
    LBM_STEP_CASE(kNone, kChannel)
    LBM_STEP_CASE(kTypeI, kChannel)
    LBM_STEP_CASE(kTypeII, kChannel)
    LBM_STEP_CASE(kTypeIII, kChannel)
    LBM_STEP_CASE(kViscous, kChannel)
#undef LBM_STEP_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbm
