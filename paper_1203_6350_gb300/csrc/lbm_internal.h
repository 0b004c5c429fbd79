// Internal declarations shared by the kernels and the C-ABI layer of liblbm.
// Not part of the public interface (include/lbm.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lbm {

// Geometry of one double-buffered population store: 9 planes of ny rows of
// `pitch` elements; plane i starts at i * plane elements from the buffer base.
struct Geometry {
    int nx, ny;
    long long pitch;  // elements per row (row bytes are a multiple of 128)
    long long plane;  // elements per plane = ny * pitch
};

// Per-lattice constants of the step, in the compute precision CT (double for
// FP64 storage, float otherwise).  All "d" quantities are deviations from the
// far-field (base) state rho0, j0 = rho0 u0.
template <typename CT>
struct StepConst {
    CT s[9];          // relaxation rates, row order of M
    CT n, m;          // Guo weights
    CT rho0, jx0, jy0;
    CT jj0;           // |j0|^2
    CT jxy0;          // jx0^2 - jy0^2
    CT pxy0;          // jx0 * jy0
    CT drf, djfx, djfy;  // reference state minus base: rho_f - rho0, j_f - j0
    CT dmeq_ref[9];   // m^eq(rho_f, j_f) - m^eq(rho0, j0), evaluated in FP64 on the host
    CT keep[9];       // (1 - s_k) / D_k: relaxation with the D^-1 of the back-transform folded in
    CT take[9];       // s_k / D_k
    CT dinv[9];       // 1 / D_k, D = diag(9, 6, 6, 36, 36, 12, 12, 4, 4)
    int bulk_x0, bulk_x1, bulk_y0, bulk_y1;  // chi = 0 for bulk_x0 <= x < bulk_x1 and bulk_y0 <= y < bulk_y1
};

// Per-axis absorbing-layer coefficients: the strength chi and the Guo factors
// 1/(1 + n chi), 1/(1 + m chi) (computed in FP64 on the host).  At a cell,
// chi = max over the two axes and, since the factors fall with chi, the
// factors are the min over the two axes.
template <typename CT>
struct alignas(4 * sizeof(CT)) AxisCoef {
    CT chi, rn, rm, pad;
};

// Host-side: the relaxation constants of StepConst for the nine rates s.
template <typename CT>
inline void fill_relax(StepConst<CT>& k, const double* s) {
    const double D[9] = {9, 6, 6, 36, 36, 12, 12, 4, 4};
    for (int i = 0; i < 9; ++i) {
        k.keep[i] = static_cast<CT>((1.0 - s[i]) / D[i]);
        k.take[i] = static_cast<CT>(s[i] / D[i]);
        k.dinv[i] = static_cast<CT>(1.0 / D[i]);
    }
}

// Host-side: the longest run [lo, hi) of zeros in a[0..n) ([0, 0) if none).
inline void zero_run(const double* a, int n, int& lo, int& hi) {
    lo = hi = 0;
    for (int i = 0; i < n;) {
        if (a[i] != 0.0) {
            ++i;
            continue;
        }
        int j = i;
        while (j < n && a[j] == 0.0) ++j;
        if (j - i > hi - lo) {
            lo = i;
            hi = j;
        }
        i = j;
    }
}

enum Storage { kF64 = 0, kF32 = 1, kF16 = 2, kBF16 = 3 };
enum Variant { kNone = 0, kTypeI = 1, kTypeII = 2, kTypeIII = 3, kViscous = 4 };
enum Bc { kDirichlet = 0, kPeriodic = 1 };

// Step launchers, one translation unit per storage type.  src holds the
// post-collision state of time t (pulled), dst receives that of time t + 1.
// pdl != 0: launch as a programmatic dependent of the previous kernel.
cudaError_t launch_step_f64(const void* src, void* dst, const Geometry& g,
                            const StepConst<double>& k, const AxisCoef<double>* tx,
                            const AxisCoef<double>* ty, int variant, int bc, cudaStream_t st,
                            int pdl);
cudaError_t launch_step_f32(const void* src, void* dst, const Geometry& g,
                            const StepConst<float>& k, const AxisCoef<float>* tx,
                            const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                            int pdl);
cudaError_t launch_step_f16(const void* src, void* dst, const Geometry& g,
                            const StepConst<float>& k, const AxisCoef<float>* tx,
                            const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                            int pdl);
cudaError_t launch_step_bf16(const void* src, void* dst, const Geometry& g,
                             const StepConst<float>& k, const AxisCoef<float>* tx,
                             const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                            int pdl);

// Base-state parameters of the auxiliary kernels (always FP64).
struct BaseState {
    double rho0, ux0, uy0;
};

// Time-0 store from FP64 fields (device pointers, [ny][nx]).
cudaError_t launch_init(int storage, void* dst, const Geometry& g, const BaseState& b,
                        const double* rho, const double* ux, const double* uy, int bc,
                        cudaStream_t st);
// Time-0 store of a Gaussian density pulse eps exp(-ln2 r^2 / b^2) centred at
// (xc, yc) on the far-field state, computed in the kernel.
cudaError_t launch_init_pulse(int storage, void* dst, const Geometry& g, const BaseState& b,
                              double eps, double half_width, double xc, double yc, int bc,
                              cudaStream_t st);
// Fields of the current time (device outputs, any may be null).
cudaError_t launch_moments(int storage, const void* src, const Geometry& g, const BaseState& b,
                           int bc, double* rho_dev, double* ux, double* uy, cudaStream_t st);
// Diagnostics: first pass writes `blocks` partial sums of kDiag doubles to
// partial[], second pass reduces them in a fixed order into out[kDiag].
constexpr int kDiag = 6;
constexpr int kDiagBlocks = 608;  // 4 per SM on a 152-SM GB300
cudaError_t launch_diagnostics(int storage, const void* src, const Geometry& g,
                               const BaseState& b, int bc, int x0, int y0, int x1, int y1,
                               double* partial, double* out, cudaStream_t st);

// Bytes per stored population.
inline size_t storage_bytes(int storage) {
    return storage == kF64 ? 8 : storage == kF32 ? 4 : 2;
}

}  // namespace lbm
