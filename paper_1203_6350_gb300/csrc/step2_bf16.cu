// Two-cells-per-thread step kernels for __nv_bfloat16 population storage (packed FP32 compute).
#include "lbm_step2.cuh"

namespace lbm {

cudaError_t launch_step2_bf16(const void* src, void* dst, const Geometry& g, const StepConst<F2>& k,
                           const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                           int bc, cudaStream_t st, int pdl) {
    return launch_step2_t<__nv_bfloat16>(src, dst, g, k, tx, ty, variant, bc, st, pdl);
}

}  // namespace lbm
