// Step kernel with compensated arithmetic: FP32 population storage, the whole
// collision (moments, rho*/j*, relaxation, damping term, back-transform) in
// float-float (ff.cuh).  The per-step rounding left is that of storing the
// populations in FP32; the FP32 kernel adds about ten roundings of its own
// per population per step, which accumulate once the field has decayed.
#include "ff.cuh"
#include "lbm_step.cuh"

namespace lbm {

template <int VAR>
__device__ __forceinline__ void collide_cell_ff(FF (&v)[9], int x, int y, const StepConst<FF>& k,
                                                const AxisCoef<float>* tx,
                                                const AxisCoef<float>* ty) {
    if (VAR == kNone || (x >= k.bulk_x0 && x < k.bulk_x1 && y >= k.bulk_y0 && y < k.bulk_y1)) {
        collide_bulk(v, k);
    } else if (VAR == kViscous) {
        const float r = fmaxf(load_coef(tx, x).chi, load_coef(ty, y).chi);
        if (r > 0.0f)
            collide_viscous(v, ff(r), k);
        else
            collide_bulk(v, k);
    } else {
        const AxisCoef<float> ax = load_coef(tx, x), ay = load_coef(ty, y);
        const float chi = fmaxf(ax.chi, ay.chi);
        if (chi > 0.0f)
            collide_layer<FF, VAR>(v, ff(chi), ff(fminf(ax.rn, ay.rn)), ff(fminf(ax.rm, ay.rm)), k);
        else
            collide_bulk(v, k);
    }
}

template <int VAR, int BC>
__global__ void __launch_bounds__(kStepBX* kStepBY)
    step_ff_kernel(PlanePtrs<float> src, PlanePtrs<float> dst, int nx, int ny, int pitch,
                   StepConst<FF> k, const AxisCoef<float>* __restrict__ tx,
                   const AxisCoef<float>* __restrict__ ty, LineSource ls) {
    const int bx0 = blockIdx.x * kStepBX, by0 = blockIdx.y * kStepBY;
    const int x = bx0 + threadIdx.x;
    const int y = by0 + threadIdx.y;
    const bool interior = bx0 > 0 && by0 > 0 && bx0 + kStepBX < nx && by0 + kStepBY < ny;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (x >= nx || y >= ny) {
        asm volatile("griddepcontrol.launch_dependents;");
        return;
    }
    const int o = y * pitch + x;
    float g[9];
    PullSites ps;
    if (interior) {
        ps.interior(pitch);
        pull_all<float, BC, false>(src, o, ps, g);
    } else {
        ps.edge<BC>(x, y, nx, ny, pitch);
        const double src_s = (BC == kChannel && x == 0) ? line_source_scale(ls) : 0.0;
        pull_all<float, BC, true>(src, o, ps, g, src_s, ls.e);
    }
    FF v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = ff(g[i]);
    collide_cell_ff<VAR>(v, x, y, k, tx, ty);
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = ff_round(v[i]);
    store_all<float>(dst, o, g);
    asm volatile("griddepcontrol.launch_dependents;");
}

cudaError_t launch_step_ff(const void* src, void* dst, const Geometry& g, const StepConst<FF>& k,
                           const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                           int bc, cudaStream_t st, int pdl, const LineSource& ls) {
    const PlanePtrs<float> s = plane_ptrs<float>(const_cast<void*>(src), g.plane);
    const PlanePtrs<float> d = plane_ptrs<float>(dst, g.plane);
    const int pitch = static_cast<int>(g.pitch);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((g.nx + kStepBX - 1) / kStepBX, (g.ny + kStepBY - 1) / kStepBY);
    cfg.blockDim = dim3(kStepBX, kStepBY);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
#define LBM_FF_CASE(V, B)                                                                     \
    if (variant == V && bc == B)                                                              \
        return cudaLaunchKernelEx(&cfg, step_ff_kernel<V, B>, s, d, g.nx, g.ny, pitch, k, tx, ty, ls);
    LBM_FF_CASE(kNone, kDirichlet)
    LBM_FF_CASE(kTypeI, kDirichlet)
    LBM_FF_CASE(kTypeII, kDirichlet)
    LBM_FF_CASE(kTypeIII, kDirichlet)
    LBM_FF_CASE(kViscous, kDirichlet)
    LBM_FF_CASE(kNone, kPeriodic)
    LBM_FF_CASE(kTypeI, kPeriodic)
    LBM_FF_CASE(kTypeII, kPeriodic)
    LBM_FF_CASE(kTypeIII, kPeriodic)
    LBM_FF_CASE(kViscous, kPeriodic)
    LBM_FF_CASE(kNone, kChannel)
    LBM_FF_CASE(kTypeI, kChannel)
    LBM_FF_CASE(kTypeII, kChannel)
    LBM_FF_CASE(kTypeIII, kChannel)
    LBM_FF_CASE(kViscous, kChannel)
#undef LBM_FF_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbm
