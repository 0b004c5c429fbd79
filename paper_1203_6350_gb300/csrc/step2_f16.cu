// Two-cells-per-thread step kernels for __half population storage (packed FP32
// compute): one step per launch, and two steps per launch (temporal blocking).
#include "lbm_step_tma.cuh"

namespace lbm {

cudaError_t launch_step2_f16(const void* src, void* dst, const Geometry& g, const StepConst<F2>& k,
                           const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                           int bc, cudaStream_t st, int pdl, const LineSource& ls) {
    return launch_step2_t<__half>(src, dst, g, k, tx, ty, variant, bc, st, pdl, ls);
}

cudaError_t launch_step_tb2_f16(const void* src, void* dst, const Geometry& g,
                              const StepConst<F2>& k, const AxisCoef<float>* tx,
                              const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                              int pdl) {
    return launch_step_tb2_t<__half>(src, dst, g, k, tx, ty, variant, bc, st, pdl);
}

cudaError_t launch_step_tb2_tma_f16(const CUtensorMap& src_map, void* dst, const Geometry& g,
                                    const StepConst<F2>& k, const AxisCoef<float>* tx,
                                    const AxisCoef<float>* ty, int variant, int grid, int* err,
                                    cudaStream_t st, int pdl, int polls) {
    return launch_step_tb2_tma<__half>(src_map, static_cast<__half*>(dst), g, k, tx, ty, variant,
                                   grid, err, st, pdl, polls);
}

cudaError_t prepare_step_tb2_tma_f16(int* per_sm) {
    return prepare_step_tb2_tma<__half>(per_sm);
}

}  // namespace lbm
