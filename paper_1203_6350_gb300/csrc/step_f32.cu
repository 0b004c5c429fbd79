// Step kernels for float population storage (compute in float).
#include "lbm_step.cuh"

namespace lbm {

cudaError_t launch_step_f32(const void* src, void* dst, const Geometry& g,
                        const StepConst<float>& k, const float* chi_x, const float* chi_y,
                        int variant, int bc, cudaStream_t st) {
    return launch_step_t<float>(src, dst, g, k, chi_x, chi_y, variant, bc, st);
}

}  // namespace lbm
