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

cudaError_t prepare_step_tb2_tma_f32(int* per_sm) { return prepare_step_tb2_tma<float>(per_sm); }

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

// elem = 4 (FP32) or 2 (FP16 / BF16 deviations, bf16 selecting the type).
bool encode_tma_map(CUtensorMap* map, void* base, const Geometry& g, int elem, bool bf16) {
    const EncodeTiled f = encode_tiled();
    if (!f || !base || (elem != 4 && elem != 2)) return false;
    const cuuint64_t dim[3] = {static_cast<cuuint64_t>(g.nx), static_cast<cuuint64_t>(g.ny), 9};
    const cuuint64_t stride[2] = {static_cast<cuuint64_t>(g.pitch) * elem,
                                  static_cast<cuuint64_t>(g.plane) * elem};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(elem == 4 ? TmaBox<float>::w
                                                                  : TmaBox<__half>::w),
                               static_cast<cuuint32_t>(TmaBox<float>::h), 9};
    const cuuint32_t step[3] = {1, 1, 1};
    const CUtensorMapDataType dt = elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : bf16    ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                             : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    // elements outside the extent read as zero (OOB fill "none"); L2 fills from DRAM in
    // 256-byte units (measured 0.6 % ahead of 128 at 4096^2, level at 16384^2 and batched)
    return f(map, dt, 3, base, dim, stride, box, step, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_tma_map_f32(CUtensorMap* map, void* base, const Geometry& g) {
    return encode_tma_map(map, base, g, 4, false);
}

}  // namespace lbm
