// Step kernels for double population storage (compute in double).
#include "lbm_step.cuh"

namespace lbm {

cudaError_t launch_step_f64(const void* src, void* dst, const Geometry& g,
                        const StepConst<double>& k, const AxisCoef<double>* tx,
                        const AxisCoef<double>* ty, int variant, int bc, cudaStream_t st, int pdl,
                        const LineSource& ls) {
    return launch_step_t<double>(src, dst, g, k, tx, ty, variant, bc, st, pdl, ls);
}

}  // namespace lbm
