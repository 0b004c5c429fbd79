// Step kernels for __half population storage (compute in float).
#include "lbm_step.cuh"

namespace lbm {

cudaError_t launch_step_f16(const void* src, void* dst, const Geometry& g,
                        const StepConst<float>& k, const AxisCoef<float>* tx,
                        const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st, int pdl,
                        const LineSource& ls) {
    return launch_step_t<__half>(src, dst, g, k, tx, ty, variant, bc, st, pdl, ls);
}

}  // namespace lbm
