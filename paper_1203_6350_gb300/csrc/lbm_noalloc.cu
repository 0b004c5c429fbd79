// lbm_diagnostics_noalloc: the diagnostics reduction for callers that cannot
// allocate device memory.  Its block partial sums live in a file-scope static
// device array instead of memory the library allocates per call or per handle.
#include <mutex>

#include "d2q9_cell.cuh"
#include "lbm.h"

namespace {

using namespace lbm;

constexpr int kNaThreads = 256;
constexpr int kNaCellsPerBlock = 16384;  // cells summed by one block
constexpr int kNaMaxBlocks = 16384;      // capacity of the static scratch, in blocks
constexpr long long kNaMaxCells = (long long)kNaCellsPerBlock * kNaMaxBlocks;  // 268,435,456
constexpr int kNaMaxDevices = 64;

// kNaMaxBlocks partial rows of kDiag sums, then the kDiag final sums: 786,480
// bytes on every device that loads this library, held until the process exits.
// Each call overwrites every slot it reads, so nothing needs clearing between
// calls; calls that overlap on the GPU share the array and race.
static __device__ __align__(256) double g_na_scratch[kNaMaxBlocks * kDiag + kDiag];

std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {};

// Device address of g_na_scratch on the current device.  Host code cannot use
// the symbol itself (on the host it names a stand-in, not device memory), so
// the address is looked up once per device, with that device current.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block b sums the cells b * kNaCellsPerBlock ... of the region taken in
// row-major order (region width w, first cell (x0, y0)).
template <typename T, int BC>
__global__ void __launch_bounds__(kNaThreads)
    na_partial_kernel(PlanePtrs<T> src, Geometry g, BaseState b, int x0, int y0, int w,
                      long long ncell, double* partial) {
    using CT = typename Codec<T>::CT;
    double acc[kDiag] = {0, 0, 0, 0, 0, 0};
    const CT rho0 = CT(b.rho0), ux0 = CT(b.ux0), uy0 = CT(b.uy0);
    const long long begin = (long long)blockIdx.x * kNaCellsPerBlock;
    const long long end = begin + kNaCellsPerBlock < ncell ? begin + kNaCellsPerBlock : ncell;
    long long c = begin + threadIdx.x;
    int ry = (int)(c / w);
    int rx = (int)(c - (long long)ry * w);
    const int pitch = static_cast<int>(g.pitch);
    // the block's stride kNaThreads, as whole rows and a remainder below w
    const int step_y = kNaThreads / w, step_x = kNaThreads - step_y * w;
    for (; c < end; c += kNaThreads) {
        const int x = x0 + rx, y = y0 + ry;
        PullSites ps;
        ps.edge<BC>(x, y, g.nx, g.ny, pitch);
        CT v[9];
        pull_all<T, BC, true>(src, y * pitch + x, ps, v);
        CT m[9];
        moments9(v, m);
        const CT r = m[0], jx = m[1], jy = m[2];
        const CT inv = CT(1) / (rho0 + r);
        const CT dux = (jx - r * ux0) * inv;  // u - u0 = (j' - rho' u0) / rho
        const CT duy = (jy - r * uy0) * inv;
        const double dr = double(r);
        acc[0] += dr;
        acc[1] += double(jx);
        acc[2] += double(jy);
        acc[3] += dr * dr / (6.0 * b.rho0) +
                  0.5 * b.rho0 * (double(dux) * double(dux) + double(duy) * double(duy));
        acc[4] += dr * dr;
        acc[5] += (isfinite(r) && isfinite(dux) && isfinite(duy)) ? 0.0 : 1.0;
        rx += step_x;
        ry += step_y;
        if (rx >= w) {
            rx -= w;
            ++ry;
        }
    }
    __shared__ double red[kDiag][kNaThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kDiag; ++q) {
        const double v = na_warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiag) {
        double s = 0.0;
        for (int k = 0; k < kNaThreads / 32; ++k) s += red[threadIdx.x][k];
        partial[blockIdx.x * kDiag + threadIdx.x] = s;
    }
}

// One block adds the partial rows in a fixed order.
__global__ void __launch_bounds__(kNaThreads)
    na_final_kernel(const double* partial, int blocks, double* out) {
    __shared__ double red[kDiag][kNaThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kDiag; ++q) {
        double s = 0.0;
        for (int k = threadIdx.x; k < blocks; k += kNaThreads) s += partial[k * kDiag + q];
        s = na_warp_sum(s);
        if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < kDiag) {
        double s = 0.0;
        for (int k = 0; k < kNaThreads / 32; ++k) s += red[threadIdx.x][k];
        out[threadIdx.x] = s;
    }
}

template <typename T>
cudaError_t na_launch(const void* state, const Geometry& g, const BaseState& b, int bc, int x0,
                      int y0, int w, long long ncell, double* partial, double* result,
                      cudaStream_t st) {
    const PlanePtrs<T> s = plane_ptrs<T>(const_cast<void*>(state), g.plane);
    const int blocks = ncell > 0 ? (int)((ncell + kNaCellsPerBlock - 1) / kNaCellsPerBlock) : 0;
    if (blocks > 0) {
        if (bc == kPeriodic)
            na_partial_kernel<T, kPeriodic><<<blocks, kNaThreads, 0, st>>>(s, g, b, x0, y0, w, ncell, partial);
        else
            na_partial_kernel<T, kDirichlet><<<blocks, kNaThreads, 0, st>>>(s, g, b, x0, y0, w, ncell, partial);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    na_final_kernel<<<1, kNaThreads, 0, st>>>(partial, blocks, result);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm_diagnostics_noalloc(const void* state, lbm_storage storage, int nx, int ny, lbm_bc bc,
                            double rho0, double ux0, double uy0, int x0, int y0, int x1, int y1,
                            double* out, int out_on_device, void* cuda_stream) {
    if (storage < LBM_F64 || storage > LBM_BF16DEV) return LBM_ERR_ARG;
    if (bc != LBM_BC_DIRICHLET_EQ && bc != LBM_BC_PERIODIC) return LBM_ERR_ARG;
    if (nx < 1 || ny < 1) return LBM_ERR_ARG;
    if (x0 < 0 || y0 < 0 || x1 > nx || y1 > ny || x0 > x1 || y0 > y1) return LBM_ERR_ARG;
    // the static scratch holds the partial sums of at most kNaMaxCells cells
    const long long ncell = (long long)(x1 - x0) * (y1 - y0);
    if (ncell > kNaMaxCells) return LBM_ERR_TOO_LARGE;
    const size_t es = storage == LBM_F64 ? 8 : storage == LBM_F32 ? 4 : 2;
    const long long pitch = (long long)((nx * es + 127) / 128 * 128 / es);
    if (pitch * ny > 2147483647LL) return LBM_ERR_TOO_LARGE;
    if (!state || !out) return LBM_ERR_ARG;
    if (!(rho0 > 0)) return LBM_ERR_ARG;

    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    double* partial = scratch;
    double* result = scratch + kNaMaxBlocks * kDiag;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const Geometry g{nx, ny, pitch, pitch * ny};
    const BaseState b{rho0, ux0, uy0};
    const int w = x1 - x0;
    double* dst = out_on_device ? out : result;
    switch (storage) {
        case LBM_F64: e = na_launch<double>(state, g, b, bc, x0, y0, w, ncell, partial, dst, st); break;
        case LBM_F32: e = na_launch<float>(state, g, b, bc, x0, y0, w, ncell, partial, dst, st); break;
        case LBM_F16DEV: e = na_launch<__half>(state, g, b, bc, x0, y0, w, ncell, partial, dst, st); break;
        default: e = na_launch<__nv_bfloat16>(state, g, b, bc, x0, y0, w, ncell, partial, dst, st); break;
    }
    if (e == cudaSuccess && !out_on_device) {
        e = cudaMemcpyAsync(out, result, kDiag * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if (!out_on_device && out[5] > 0) return LBM_ERR_NONFINITE;
    return LBM_OK;
}

}  // extern "C"
