// Step kernels for double population storage (compute in double).
#include "lbm_step.cuh"

namespace lbm {

cudaError_t launch_step_f64(const void* src, void* dst, const Geometry& g,
                        const StepConst<double>& k, const double* chi_x, const double* chi_y,
                        int variant, int bc, cudaStream_t st) {
    return launch_step_t<double>(src, dst, g, k, chi_x, chi_y, variant, bc, st);
}

}  // namespace lbm
