// Auxiliary kernels: time-0 store at equilibrium, macroscopic fields, and FP64
// diagnostics reductions.  They read the same pull-stored state as the step.
#include "d2q9_cell.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ double weight(int i) { return i == 0 ? 4.0 / 9.0 : i < 5 ? 1.0 / 9.0 : 1.0 / 36.0; }

// f^eq_i(rho, u) - f^eq_i(rho0, u0) in FP64 (the second-order D2Q9 equilibrium).
__device__ __forceinline__ double feq_dev(int i, double rho, double ux, double uy, const BaseState& b) {
    const double cu = cx(i) * ux + cy(i) * uy;
    const double cu0 = cx(i) * b.ux0 + cy(i) * b.uy0;
    const double p = rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy));
    const double p0 = b.rho0 * (1.0 + 3.0 * cu0 + 4.5 * cu0 * cu0 - 1.5 * (b.ux0 * b.ux0 + b.uy0 * b.uy0));
    return weight(i) * (p - p0);
}

template <typename T, int I>
__device__ __forceinline__ void init_plane(T* dst, const Geometry& g, const BaseState& b,
                                           const double* rho, const double* ux, const double* uy,
                                           int bc, int x, int y) {
    // The pull at cell (x, y) + c_I reads this slot, so it holds f^eq there.
    int sx = x + cx(I), sy = y + cy(I);
    bool ok = sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny;
    if (!ok && bc == kPeriodic) {
        sx = (sx + g.nx) % g.nx;
        sy = (sy + g.ny) % g.ny;
        ok = true;
    }
    double v = 0.0;
    if (ok) {
        const long long c = (long long)sy * g.nx + sx;
        v = feq_dev(I, rho[c], ux[c], uy[c], b);
    }
    using CT = typename Codec<T>::CT;
    dst[I * g.plane + (long long)y * g.pitch + x] = Codec<T>::template enc<I>(static_cast<CT>(v));
}

template <typename T>
__global__ void init_kernel(T* dst, Geometry g, BaseState b, const double* rho, const double* ux,
                            const double* uy, int bc) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    init_plane<T, 0>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 1>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 2>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 3>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 4>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 5>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 6>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 7>(dst, g, b, rho, ux, uy, bc, x, y);
    init_plane<T, 8>(dst, g, b, rho, ux, uy, bc, x, y);
}

// rho', j' of the pulled populations at (x, y), accumulated in FP64.
template <typename T, int BC>
__device__ __forceinline__ void cell_moments(const T* src, const Geometry& g, int x, int y,
                                             double& r, double& jx, double& jy) {
    using CT = typename Codec<T>::CT;
    PullSites ps;
    ps.init<BC>(x, y, g);
    CT v[9];
    pull_all<T, BC>(src, g.plane, (long long)y * g.pitch + x, ps, v);
    r = 0.0;
    jx = 0.0;
    jy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double d = static_cast<double>(v[i]);
        r += d;
        jx += cx(i) * d;
        jy += cy(i) * d;
    }
}

template <typename T, int BC>
__global__ void moments_kernel(const T* src, Geometry g, BaseState b, double* rho_dev, double* ux,
                               double* uy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    double r, jx, jy;
    cell_moments<T, BC>(src, g, x, y, r, jx, jy);
    const long long c = (long long)y * g.nx + x;
    const double rho = b.rho0 + r;
    if (rho_dev) rho_dev[c] = r;
    if (ux) ux[c] = (b.rho0 * b.ux0 + jx) / rho;
    if (uy) uy[c] = (b.rho0 * b.uy0 + jy) / rho;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kDiagThreads = 256;

// First pass: each block strides over the region's cells in a fixed order and
// writes its kDiag partial sums.
template <typename T, int BC>
__global__ void __launch_bounds__(kDiagThreads)
    diag_partial_kernel(const T* src, Geometry g, BaseState b, int x0, int y0, int x1, int y1,
                        double* partial) {
    const long long w = x1 - x0;
    const long long ncell = w * (long long)(y1 - y0);
    double acc[kDiag] = {0, 0, 0, 0, 0, 0};
    const double cs2 = 1.0 / 3.0;
    for (long long c = (long long)blockIdx.x * kDiagThreads + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * kDiagThreads) {
        const int x = x0 + (int)(c % w);
        const int y = y0 + (int)(c / w);
        double r, jx, jy;
        cell_moments<T, BC>(src, g, x, y, r, jx, jy);
        const double rho = b.rho0 + r;
        // u - u0 = (j' - rho' u0) / rho, with j' = j - rho0 u0
        const double dux = (jx - r * b.ux0) / rho;
        const double duy = (jy - r * b.uy0) / rho;
        const double e = cs2 * r * r / (2.0 * b.rho0) + 0.5 * b.rho0 * (dux * dux + duy * duy);
        const bool finite = isfinite(r) && isfinite(dux) && isfinite(duy);
        acc[0] += r;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += e;
        acc[4] += r * r;
        acc[5] += finite ? 0.0 : 1.0;
    }
    __shared__ double red[kDiag][kDiagThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kDiag; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiag) {
        double s = 0.0;
        for (int k = 0; k < kDiagThreads / 32; ++k) s += red[threadIdx.x][k];
        partial[(long long)blockIdx.x * kDiag + threadIdx.x] = s;
    }
}

// Second pass: one block adds the partials in a fixed order.
__global__ void __launch_bounds__(kDiagThreads)
    diag_final_kernel(const double* partial, int blocks, double* out) {
    __shared__ double red[kDiag][kDiagThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kDiag; ++q) {
        double s = 0.0;
        for (int k = threadIdx.x; k < blocks; k += kDiagThreads) s += partial[(long long)k * kDiag + q];
        s = warp_sum(s);
        if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < kDiag) {
        double s = 0.0;
        for (int k = 0; k < kDiagThreads / 32; ++k) s += red[threadIdx.x][k];
        out[threadIdx.x] = s;
    }
}

template <typename T>
cudaError_t init_t(void* dst, const Geometry& g, const BaseState& b, const double* rho,
                   const double* ux, const double* uy, int bc, cudaStream_t st) {
    const dim3 block(128, 2), grid((g.nx + 127) / 128, (g.ny + 1) / 2);
    init_kernel<T><<<grid, block, 0, st>>>(static_cast<T*>(dst), g, b, rho, ux, uy, bc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t moments_t(const void* src, const Geometry& g, const BaseState& b, int bc, double* r,
                      double* ux, double* uy, cudaStream_t st) {
    const dim3 block(128, 2), grid((g.nx + 127) / 128, (g.ny + 1) / 2);
    const T* s = static_cast<const T*>(src);
    if (bc == kPeriodic)
        moments_kernel<T, kPeriodic><<<grid, block, 0, st>>>(s, g, b, r, ux, uy);
    else
        moments_kernel<T, kDirichlet><<<grid, block, 0, st>>>(s, g, b, r, ux, uy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t diag_t(const void* src, const Geometry& g, const BaseState& b, int bc, int x0, int y0,
                   int x1, int y1, double* partial, double* out, cudaStream_t st) {
    const T* s = static_cast<const T*>(src);
    if (bc == kPeriodic)
        diag_partial_kernel<T, kPeriodic><<<kDiagBlocks, kDiagThreads, 0, st>>>(s, g, b, x0, y0, x1, y1, partial);
    else
        diag_partial_kernel<T, kDirichlet><<<kDiagBlocks, kDiagThreads, 0, st>>>(s, g, b, x0, y0, x1, y1, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, kDiagThreads, 0, st>>>(partial, kDiagBlocks, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init(int storage, void* dst, const Geometry& g, const BaseState& b,
                        const double* rho, const double* ux, const double* uy, int bc,
                        cudaStream_t st) {
    switch (storage) {
        case kF64: return init_t<double>(dst, g, b, rho, ux, uy, bc, st);
        case kF32: return init_t<float>(dst, g, b, rho, ux, uy, bc, st);
        case kF16: return init_t<__half>(dst, g, b, rho, ux, uy, bc, st);
        case kBF16: return init_t<__nv_bfloat16>(dst, g, b, rho, ux, uy, bc, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_moments(int storage, const void* src, const Geometry& g, const BaseState& b,
                           int bc, double* rho_dev, double* ux, double* uy, cudaStream_t st) {
    switch (storage) {
        case kF64: return moments_t<double>(src, g, b, bc, rho_dev, ux, uy, st);
        case kF32: return moments_t<float>(src, g, b, bc, rho_dev, ux, uy, st);
        case kF16: return moments_t<__half>(src, g, b, bc, rho_dev, ux, uy, st);
        case kBF16: return moments_t<__nv_bfloat16>(src, g, b, bc, rho_dev, ux, uy, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_diagnostics(int storage, const void* src, const Geometry& g,
                               const BaseState& b, int bc, int x0, int y0, int x1, int y1,
                               double* partial, double* out, cudaStream_t st) {
    switch (storage) {
        case kF64: return diag_t<double>(src, g, b, bc, x0, y0, x1, y1, partial, out, st);
        case kF32: return diag_t<float>(src, g, b, bc, x0, y0, x1, y1, partial, out, st);
        case kF16: return diag_t<__half>(src, g, b, bc, x0, y0, x1, y1, partial, out, st);
        case kBF16: return diag_t<__nv_bfloat16>(src, g, b, bc, x0, y0, x1, y1, partial, out, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
