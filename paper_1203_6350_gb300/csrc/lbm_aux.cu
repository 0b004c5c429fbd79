// Auxiliary kernels: time-0 store at equilibrium, macroscopic fields, and FP64
// diagnostics reductions.  They read the same pull-stored state as the step.
#include "d2q9_cell.cuh"

namespace lbm {

namespace {

template <typename CT>
__device__ __forceinline__ CT weight(int i) {
    return i == 0 ? CT(4) / CT(9) : i < 5 ? CT(1) / CT(9) : CT(1) / CT(36);
}

// f^eq_i(rho, u) - f^eq_i(rho0, u0) of the second-order D2Q9 equilibrium, from
// rho' = rho - rho0 and du = u - u0 without cancellation:
//   w_i [rho' (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
//        + rho0 (3 c.du + 9/2 (c.du)(c.u + c.u0) - 3/2 du.(u + u0))].
template <typename CT>
__device__ __forceinline__ CT feq_dev(int i, CT dr, CT ux, CT uy, CT dux, CT duy, CT rho0, CT ux0,
                                      CT uy0) {
    const CT cu = cx(i) * ux + cy(i) * uy;
    const CT cu0 = cx(i) * ux0 + cy(i) * uy0;
    const CT cdu = cx(i) * dux + cy(i) * duy;
    const CT a = CT(1) + CT(3) * cu + CT(4.5) * cu * cu - CT(1.5) * (ux * ux + uy * uy);
    const CT b = CT(3) * cdu + CT(4.5) * cdu * (cu + cu0) - CT(1.5) * (dux * (ux + ux0) + duy * (uy + uy0));
    return weight<CT>(i) * (dr * a + rho0 * b);
}

template <typename T, int I>
__device__ __forceinline__ void init_plane(const PlanePtrs<T>& dst, const Geometry& g,
                                           const BaseState& b, const double* rho, const double* ux,
                                           const double* uy, int bc, int x, int y) {
    using CT = typename Codec<T>::CT;
    // The pull at cell (x, y) + c_I reads this slot, so it holds f^eq there.
    int sx = x + cx(I), sy = y + cy(I);
    if (bc == kChannel) sy = (sy + g.ny) % g.ny;  // periodic in y only
    bool ok = sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny;
    if (!ok && bc == kPeriodic) {
        sx = (sx + g.nx) % g.nx;
        sy = (sy + g.ny) % g.ny;
        ok = true;
    }
    CT v = CT(0);
    if (ok) {
        const long long c = (long long)sy * g.nx + sx;
        const double u = ux[c], w = uy[c];
        v = feq_dev<CT>(I, CT(rho[c] - b.rho0), CT(u), CT(w), CT(u - b.ux0), CT(w - b.uy0),
                        CT(b.rho0), CT(b.ux0), CT(b.uy0));
    }
    dst.p[I][(long long)y * g.pitch + x] = Codec<T>::template enc<I>(v);
}

template <typename T>
__global__ void init_kernel(PlanePtrs<T> dst, Geometry g, BaseState b, const double* rho,
                            const double* ux, const double* uy, int bc) {
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

// Time 0 of the acoustic pulse of Sec. 4.1 (Eqs. pulseprofile, 3:para0) without
// any input field: rho = rho0 + eps exp(-alpha |x - x_c|^2), u = u0 at every cell.
template <typename T, int I>
__device__ __forceinline__ void pulse_plane(const PlanePtrs<T>& dst, const Geometry& g,
                                            const BaseState& b, double eps, double alpha,
                                            double xc, double yc, int bc, int x, int y) {
    using CT = typename Codec<T>::CT;
    int sx = x + cx(I), sy = y + cy(I);
    if (bc == kChannel) sy = (sy + g.ny) % g.ny;  // periodic in y only
    bool ok = sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny;
    if (!ok && bc == kPeriodic) {
        sx = (sx + g.nx) % g.nx;
        sy = (sy + g.ny) % g.ny;
        ok = true;
    }
    CT v = CT(0);
    if (ok) {
        const double dx = sx - xc, dy = sy - yc;
        const double dr = eps * exp(-alpha * (dx * dx + dy * dy));
        v = feq_dev<CT>(I, CT(dr), CT(b.ux0), CT(b.uy0), CT(0), CT(0), CT(b.rho0), CT(b.ux0),
                        CT(b.uy0));
    }
    dst.p[I][(long long)y * g.pitch + x] = Codec<T>::template enc<I>(v);
}

template <typename T>
__global__ void pulse_kernel(PlanePtrs<T> dst, Geometry g, BaseState b, double eps, double alpha,
                             double xc, double yc, int bc) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    pulse_plane<T, 0>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 1>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 2>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 3>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 4>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 5>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 6>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 7>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
    pulse_plane<T, 8>(dst, g, b, eps, alpha, xc, yc, bc, x, y);
}

template <typename T>
cudaError_t pulse_t(void* dst, const Geometry& g, const BaseState& b, double eps, double alpha,
                    double xc, double yc, int bc, cudaStream_t st) {
    const dim3 block(128, 2), grid((g.nx + 127) / 128, (g.ny + 1) / 2);
    pulse_kernel<T><<<grid, block, 0, st>>>(plane_ptrs<T>(dst, g.plane), g, b, eps, alpha, xc, yc, bc);
    return cudaGetLastError();
}

// rho', j' of the pulled populations at (x, y), summed in the compute precision.
template <typename T, int BC>
__device__ __forceinline__ void cell_moments(const PlanePtrs<T>& src, const Geometry& g, int x,
                                             int y, typename Codec<T>::CT& r,
                                             typename Codec<T>::CT& jx,
                                             typename Codec<T>::CT& jy, const LineSource& ls) {
    using CT = typename Codec<T>::CT;
    PullSites ps;
    ps.edge<BC>(x, y, g.nx, g.ny, static_cast<int>(g.pitch));
    CT v[9];
    const double src_s = (BC == kChannel && x == 0) ? line_source_scale(ls) : 0.0;
    pull_all<T, BC, true>(src, y * static_cast<int>(g.pitch) + x, ps, v, src_s, ls.e);
    CT m[9];
    moments9(v, m);
    r = m[0];
    jx = m[1];
    jy = m[2];
}

template <typename T, int BC>
__global__ void moments_kernel(PlanePtrs<T> src, Geometry g, BaseState b, double* rho_dev,
                               double* ux, double* uy, LineSource ls) {
    using CT = typename Codec<T>::CT;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    CT r, jx, jy;
    cell_moments<T, BC>(src, g, x, y, r, jx, jy, ls);
    const long long c = (long long)y * g.nx + x;
    const double rho = b.rho0 + double(r);
    if (rho_dev) rho_dev[c] = double(r);
    if (ux) ux[c] = (b.rho0 * b.ux0 + double(jx)) / rho;
    if (uy) uy[c] = (b.rho0 * b.uy0 + double(jy)) / rho;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kDiagThreads = 256;

// First pass: block (bx, by) of a gx x gy grid takes the rows y0 + by, + gy, ...
// and the columns x0 + bx * 256 + t, + gx * 256, ... of the region, and writes
// its kDiag sums (FP64) to partial[by * gx + bx].
template <typename T, int BC>
__global__ void __launch_bounds__(kDiagThreads)
    diag_partial_kernel(PlanePtrs<T> src, Geometry g, BaseState b, int x0, int y0, int x1, int y1,
                        double* partial, LineSource ls) {
    using CT = typename Codec<T>::CT;
    double acc[kDiag] = {0, 0, 0, 0, 0, 0};
    const CT rho0 = CT(b.rho0), ux0 = CT(b.ux0), uy0 = CT(b.uy0);
    for (int y = y0 + blockIdx.y; y < y1; y += gridDim.y) {
        for (int x = x0 + blockIdx.x * kDiagThreads + threadIdx.x; x < x1;
             x += gridDim.x * kDiagThreads) {
            CT r, jx, jy;
            cell_moments<T, BC>(src, g, x, y, r, jx, jy, ls);
            // u - u0 = (j' - rho' u0) / rho, with j' = j - rho0 u0
            const CT inv = CT(1) / (rho0 + r);
            const CT dux = (jx - r * ux0) * inv;
            const CT duy = (jy - r * uy0) * inv;
            const double dr = double(r);
            const double e = dr * dr / (6.0 * b.rho0) +
                             0.5 * b.rho0 * (double(dux) * double(dux) + double(duy) * double(duy));
            const bool finite = isfinite(r) && isfinite(dux) && isfinite(duy);
            acc[0] += dr;
            acc[1] += double(jx);
            acc[2] += double(jy);
            acc[3] += e;
            acc[4] += dr * dr;
            acc[5] += finite ? 0.0 : 1.0;
        }
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
        partial[(blockIdx.y * gridDim.x + blockIdx.x) * kDiag + threadIdx.x] = s;
    }
}

// Second pass: one block adds the partials in a fixed order.
__global__ void __launch_bounds__(kDiagThreads)
    diag_final_kernel(const double* partial, int blocks, double* out) {
    __shared__ double red[kDiag][kDiagThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kDiag; ++q) {
        double s = 0.0;
        for (int k = threadIdx.x; k < blocks; k += kDiagThreads) s += partial[k * kDiag + q];
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
    init_kernel<T><<<grid, block, 0, st>>>(plane_ptrs<T>(dst, g.plane), g, b, rho, ux, uy, bc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t moments_t(const void* src, const Geometry& g, const BaseState& b, int bc, double* r,
                      double* ux, double* uy, cudaStream_t st, const LineSource& ls) {
    const dim3 block(128, 2), grid((g.nx + 127) / 128, (g.ny + 1) / 2);
    const PlanePtrs<T> s = plane_ptrs<T>(const_cast<void*>(src), g.plane);
    if (bc == kPeriodic)
        moments_kernel<T, kPeriodic><<<grid, block, 0, st>>>(s, g, b, r, ux, uy, ls);
    else if (bc == kChannel)
        moments_kernel<T, kChannel><<<grid, block, 0, st>>>(s, g, b, r, ux, uy, ls);
    else
        moments_kernel<T, kDirichlet><<<grid, block, 0, st>>>(s, g, b, r, ux, uy, ls);
    return cudaGetLastError();
}

template <typename T>
cudaError_t diag_t(const void* src, const Geometry& g, const BaseState& b, int bc, int x0, int y0,
                   int x1, int y1, double* partial, double* out, cudaStream_t st,
                   const LineSource& ls) {
    const PlanePtrs<T> s = plane_ptrs<T>(const_cast<void*>(src), g.plane);
    const int w = x1 - x0, h = y1 - y0;
    const int gx = w <= 0 ? 1 : (w + kDiagThreads - 1) / kDiagThreads < 4 ? (w + kDiagThreads - 1) / kDiagThreads : 4;
    int gy = kDiagBlocks / gx;
    if (h > 0 && h < gy) gy = h;
    if (gy < 1) gy = 1;
    const dim3 grid(gx, gy);
    if (bc == kPeriodic)
        diag_partial_kernel<T, kPeriodic><<<grid, kDiagThreads, 0, st>>>(s, g, b, x0, y0, x1, y1, partial, ls);
    else if (bc == kChannel)
        diag_partial_kernel<T, kChannel><<<grid, kDiagThreads, 0, st>>>(s, g, b, x0, y0, x1, y1, partial, ls);
    else
        diag_partial_kernel<T, kDirichlet><<<grid, kDiagThreads, 0, st>>>(s, g, b, x0, y0, x1, y1, partial, ls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, kDiagThreads, 0, st>>>(partial, gx * gy, out);
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

cudaError_t launch_init_pulse(int storage, void* dst, const Geometry& g, const BaseState& b,
                              double eps, double half_width, double xc, double yc, int bc,
                              cudaStream_t st) {
    const double alpha = 0.69314718055994530942 / (half_width * half_width);  // ln 2 / b^2
    switch (storage) {
        case kF64: return pulse_t<double>(dst, g, b, eps, alpha, xc, yc, bc, st);
        case kF32: return pulse_t<float>(dst, g, b, eps, alpha, xc, yc, bc, st);
        case kF16: return pulse_t<__half>(dst, g, b, eps, alpha, xc, yc, bc, st);
        case kBF16: return pulse_t<__nv_bfloat16>(dst, g, b, eps, alpha, xc, yc, bc, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_moments(int storage, const void* src, const Geometry& g, const BaseState& b,
                           int bc, double* rho_dev, double* ux, double* uy, cudaStream_t st,
                           const LineSource& ls) {
    switch (storage) {
        case kF64: return moments_t<double>(src, g, b, bc, rho_dev, ux, uy, st, ls);
        case kF32: return moments_t<float>(src, g, b, bc, rho_dev, ux, uy, st, ls);
        case kF16: return moments_t<__half>(src, g, b, bc, rho_dev, ux, uy, st, ls);
        case kBF16: return moments_t<__nv_bfloat16>(src, g, b, bc, rho_dev, ux, uy, st, ls);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_diagnostics(int storage, const void* src, const Geometry& g,
                               const BaseState& b, int bc, int x0, int y0, int x1, int y1,
                               double* partial, double* out, cudaStream_t st,
                               const LineSource& ls) {
    switch (storage) {
        case kF64: return diag_t<double>(src, g, b, bc, x0, y0, x1, y1, partial, out, st, ls);
        case kF32: return diag_t<float>(src, g, b, bc, x0, y0, x1, y1, partial, out, st, ls);
        case kF16: return diag_t<__half>(src, g, b, bc, x0, y0, x1, y1, partial, out, st, ls);
        case kBF16: return diag_t<__nv_bfloat16>(src, g, b, bc, x0, y0, x1, y1, partial, out, st, ls);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
