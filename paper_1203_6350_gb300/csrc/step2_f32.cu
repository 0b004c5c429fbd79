// Two-cells-per-thread step kernels for float population storage (packed FP32
// compute): one step per launch, and two steps per launch (temporal blocking),
// the latter also with the tile's input staged by TMA.
#include "lbm_step_tma.cuh"

namespace lbm {

cudaError_t launch_step2_f32(const void* src, void* dst, const Geometry& g, const StepConst<F2>& k,
                           const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                           int bc, cudaStream_t st, int pdl, const LineSource& ls) {
    return launch_step2_t<float>(src, dst, g, k, tx, ty, variant, bc, st, pdl, ls);
}

cudaError_t launch_step_tb2_f32(const void* src, void* dst, const Geometry& g,
                              const StepConst<F2>& k, const AxisCoef<float>* tx,
                              const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                              int pdl) {
    return launch_step_tb2_t<float>(src, dst, g, k, tx, ty, variant, bc, st, pdl);
}

cudaError_t launch_step_tb2_tma_f32(const CUtensorMap& src_map, void* dst, const Geometry& g,
                                   const StepConst<F2>& k, const AxisCoef<float>* tx,
                                   const AxisCoef<float>* ty, int variant, int grid, int* err,
                                   cudaStream_t st, int pdl, int polls) {
    return launch_step_tb2_tma(src_map, static_cast<float*>(dst), g, k, tx, ty, variant, grid, err,
                               st, pdl, polls);
}

cudaError_t prepare_step_tb2_tma_f32(int* per_sm) { return prepare_step_tb2_tma(per_sm); }

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's cuTensorMapEncodeTiled (through the runtime, no libcuda link).
EncodeTiled encode_tiled() {
    static const EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return static_cast<EncodeTiled>(nullptr);
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}
}  // namespace

bool encode_tma_map_f32(CUtensorMap* map, void* base, const Geometry& g) {
    const EncodeTiled f = encode_tiled();
    if (!f || !base) return false;
    const cuuint64_t dim[3] = {static_cast<cuuint64_t>(g.nx), static_cast<cuuint64_t>(g.ny), 9};
    const cuuint64_t stride[2] = {static_cast<cuuint64_t>(g.pitch) * sizeof(float),
                                  static_cast<cuuint64_t>(g.plane) * sizeof(float)};
    const cuuint32_t box[3] = {kTmaW, kTmaH, 9};
    const cuuint32_t step[3] = {1, 1, 1};
    // elements outside the extent read as zero (OOB fill "none")
    return f(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dim, stride, box, step,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbm
