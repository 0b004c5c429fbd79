// Internal declarations shared by the kernels and the C-ABI layer of liblbm.
// Not part of the public interface (include/lbm.h is).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include <cuda.h>
#include <cuda_runtime.h>

namespace lbm {

// Geometry of one double-buffered population store: 9 planes of ny rows of
// `pitch` elements; plane i starts at i * plane elements from the buffer base.
struct Geometry {
    int nx, ny;
    long long pitch;  // elements per row (row bytes are a multiple of 128)
    long long plane;  // elements per plane = ny * pitch
};

// Two FP32 values packed in one 64-bit register: the populations of two
// neighbouring cells (x, x + 1) stepped together with the packed FP32
// instructions of sm_100-class GPUs (lo = cell x, hi = cell x + 1).
struct alignas(8) F2 {
    unsigned long long u;
};

// A float-float value h + l (|l| <= half an ulp of h): about 48 significant
// bits carried in two FP32 registers, for the compensated-arithmetic step
// (FP32 storage, collision in float-float; GB300's FP32 pipes are many times
// faster than its FP64 ones).
struct FF {
    float h, l;
};

// Host-side conversion of an FP64 constant to the compute type.
template <typename CT>
inline CT to_ct(double v) {
    return static_cast<CT>(v);
}
template <>
inline F2 to_ct<F2>(double v) {
    const float f = static_cast<float>(v);
    unsigned w;
    std::memcpy(&w, &f, sizeof w);
    return F2{(static_cast<unsigned long long>(w) << 32) | w};
}

template <>
inline FF to_ct<FF>(double v) {
    const float h = static_cast<float>(v);
    return FF{h, static_cast<float>(v - static_cast<double>(h))};
}

// Per-lattice constants of the step, in the compute type CT (double for FP64
// storage, float otherwise, F2 -- every constant duplicated -- for the kernel
// that steps two cells per thread).  All "d" quantities are deviations from
// the far-field (base) state rho0, j0 = rho0 u0.
//
// The relaxation of row k is written on the scaled moment a_k = m_k^+ / D_k
// that the back-transform M^T consumes (D = diag(9, 6, 6, 36, 36, 12, 12, 4, 4)):
//   a_k = keep_k m_k + take_k E_k + dinv_k chi T_k,
// with E_k the equilibrium source of the row: m_k^eq itself, except rows 5
// and 6 whose equilibrium is -j_x, -j_y; there E_k = j and take_k carries the
// minus sign.
template <typename CT>
struct StepConst {
    CT s[9];          // relaxation rates, row order of M
    // 1 - s_k.  No D2Q9 kernel reads it now; taking it out shifted the later
    // constants in the kernels' parameter block and made the 1024^2 one-step
    // kernel 1.9 % slower (44 registers instead of 46, other constant loads).
    CT oms[9];
    CT keep[9];       // (1 - s_k) / D_k
    CT take[9];       // s_k / D_k (negated for rows 5, 6)
    CT dinv[9];       // 1 / D_k
    CT dinv_lo[3];    // 1 / D_k - dinv[k] of the conserved rows, so that their scaling is unbiased
    CT rho0, jx0, jy0;
    CT jx0_2, jy0_2;  // 2 j0
    CT njj0;          // -|j0|^2
    CT njxy0;         // -(jx0^2 - jy0^2)
    CT npxy0;         // -jx0 jy0
    CT drf, djfx, djfy;   // reference state minus base: rho_f - rho0, j_f - j0
    CT ndrf, mdjfx, mdjfy;  // Guo source numerators n drf, m djfx, m djfy
    CT dmeq_ref[9];   // m^eq(rho_f, j_f) - m^eq(rho0, j0), evaluated in FP64 on the host
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

// Moment equilibria m^eq(rho, j) of the second-order D2Q9 equilibrium, in the
// row order of M (App. A.1), in FP64.
inline void moment_eq(double rho, double jx, double jy, double out[9]) {
    const double q = (jx * jx + jy * jy) / rho;
    out[0] = rho;
    out[1] = jx;
    out[2] = jy;
    out[3] = -2.0 * rho + 3.0 * q;
    out[4] = rho - 3.0 * q;
    out[5] = -jx;
    out[6] = -jy;
    out[7] = (jx * jx - jy * jy) / rho;
    out[8] = jx * jy / rho;
}

// Host-side: every constant of the step for rates s, Guo weights n, m, base
// state (rho0, u0), reference state (rho_f, u_f) and the chi = 0 rectangle
// bulk = {x0, x1, y0, y1}.  Computed in FP64, rounded once to CT.
template <typename CT>
inline StepConst<CT> make_step_const(const double* s, double n, double m, double rho0,
                                     double ux0, double uy0, double rho_f, double ux_f,
                                     double uy_f, const int* bulk) {
    StepConst<CT> k{};
    const double D[9] = {9, 6, 6, 36, 36, 12, 12, 4, 4};
    for (int i = 0; i < 9; ++i) {
        const double sign = (i == 5 || i == 6) ? -1.0 : 1.0;
        k.s[i] = to_ct<CT>(s[i]);
        k.oms[i] = to_ct<CT>(1.0 - s[i]);
        k.keep[i] = to_ct<CT>((1.0 - s[i]) / D[i]);
        k.take[i] = to_ct<CT>(sign * s[i] / D[i]);
        k.dinv[i] = to_ct<CT>(1.0 / D[i]);
    }
    // 9 fl(1/9) and 6 fl(1/6) differ from 1 by 7.5e-9 and 3.0e-8 in FP32: applied
    // every step to rho' and j', that drift grows linearly in time.  The residual
    // makes a_k = m_k / D_k of rows 0-2 correctly rounded (zero in FP64).
    for (int i = 0; i < 3; ++i) {
        const float hi = static_cast<float>(1.0 / D[i]);
        k.dinv_lo[i] = to_ct<CT>(std::is_same<CT, double>::value || std::is_same<CT, FF>::value
                                     ? 0.0
                                     : 1.0 / D[i] - hi);
    }
    const double jx0 = rho0 * ux0, jy0 = rho0 * uy0;
    k.rho0 = to_ct<CT>(rho0);
    k.jx0 = to_ct<CT>(jx0);
    k.jy0 = to_ct<CT>(jy0);
    k.jx0_2 = to_ct<CT>(2.0 * jx0);
    k.jy0_2 = to_ct<CT>(2.0 * jy0);
    k.njj0 = to_ct<CT>(-(jx0 * jx0 + jy0 * jy0));
    k.njxy0 = to_ct<CT>(-(jx0 * jx0 - jy0 * jy0));
    k.npxy0 = to_ct<CT>(-(jx0 * jy0));
    const double jfx = rho_f * ux_f, jfy = rho_f * uy_f;
    k.drf = to_ct<CT>(rho_f - rho0);
    k.djfx = to_ct<CT>(jfx - jx0);
    k.djfy = to_ct<CT>(jfy - jy0);
    k.ndrf = to_ct<CT>(n * (rho_f - rho0));
    k.mdjfx = to_ct<CT>(m * (jfx - jx0));
    k.mdjfy = to_ct<CT>(m * (jfy - jy0));
    double mr[9], mb[9];
    moment_eq(rho_f, jfx, jfy, mr);
    moment_eq(rho0, jx0, jy0, mb);
    for (int i = 0; i < 9; ++i) k.dmeq_ref[i] = to_ct<CT>(mr[i] - mb[i]);
    k.bulk_x0 = bulk[0];
    k.bulk_x1 = bulk[1];
    k.bulk_y0 = bulk[2];
    k.bulk_y1 = bulk[3];
    return k;
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
// Boundary: Dirichlet far field; periodic in both axes; channel (the line
// source of Sec. 4.2: source on the left edge, outflow on the right, periodic
// in y).
enum Bc { kDirichlet = 0, kPeriodic = 1, kChannel = 2 };

// The line source of the channel boundary.  The populations entering at the
// left edge are those of the source column's equilibrium at the time of the
// post-collision state they leave; as deviations from the base state they are
// amp sin(omega t + phase) e_i with e_i = f^eq_i(1, u0) (the equilibrium is
// linear in rho at fixed u).  A pull that yields the state of time tau uses
// t = tau - 1, tau = (time ? *time : 0) + t_off.
struct LineSource {
    const long long* time;  // device step counter (or nullptr)
    long long t_off;
    double amp, omega, phase;
    double e[9];
    const double* table;    // device: scales of the steps time .. time + n - 1 (or nullptr)
    const float* pop;       // device: float(scale * e_i) of those steps, 9 per step (or nullptr)
};

// Source deviation scale of the state that a pull with source `s` yields.
__host__ __device__ inline double line_source_scale(const LineSource& s) {
#ifdef __CUDA_ARCH__
    if (s.table) return s.table[s.t_off];  // filled by source_table_kernel for this chunk
    const long long tau = (s.time ? *s.time : 0) + s.t_off;
#else
    const long long tau = s.t_off;
#endif
    return s.amp * sin(s.omega * (double)(tau - 1) + s.phase);
}

// Step launchers, one translation unit per storage type.  src holds the
// post-collision state of time t (pulled), dst receives that of time t + 1.
// pdl != 0: launch as a programmatic dependent of the previous kernel.
cudaError_t launch_step_f64(const void* src, void* dst, const Geometry& g,
                            const StepConst<double>& k, const AxisCoef<double>* tx,
                            const AxisCoef<double>* ty, int variant, int bc, cudaStream_t st,
                            int pdl, const LineSource& ls);
cudaError_t launch_step_f32(const void* src, void* dst, const Geometry& g,
                            const StepConst<float>& k, const AxisCoef<float>* tx,
                            const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                            int pdl, const LineSource& ls);
// FP32 storage, collision in float-float (compensated arithmetic).
cudaError_t launch_step_ff(const void* src, void* dst, const Geometry& g, const StepConst<FF>& k,
                           const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                           int bc, cudaStream_t st, int pdl, const LineSource& ls);
cudaError_t launch_step_f16(const void* src, void* dst, const Geometry& g,
                            const StepConst<float>& k, const AxisCoef<float>* tx,
                            const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                            int pdl, const LineSource& ls);
cudaError_t launch_step_bf16(const void* src, void* dst, const Geometry& g,
                             const StepConst<float>& k, const AxisCoef<float>* tx,
                             const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                             int pdl, const LineSource& ls);

// Two-cells-per-thread step launchers (FP32 and 16-bit storage; packed FP32
// compute).  cudaErrorInvalidValue when 9 planes exceed 2^32 elements.
cudaError_t launch_step2_f32(const void* src, void* dst, const Geometry& g, const StepConst<F2>& k,
                             const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                             int bc, cudaStream_t st, int pdl, const LineSource& ls);
cudaError_t launch_step2_f16(const void* src, void* dst, const Geometry& g, const StepConst<F2>& k,
                             const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                             int bc, cudaStream_t st, int pdl, const LineSource& ls);
cudaError_t launch_step2_bf16(const void* src, void* dst, const Geometry& g, const StepConst<F2>& k,
                              const AxisCoef<float>* tx, const AxisCoef<float>* ty, int variant,
                              int bc, cudaStream_t st, int pdl, const LineSource& ls);

// Two steps per launch (temporal blocking through shared memory) on the
// two-cells-per-thread arithmetic: src holds time t, dst receives t + 2.
cudaError_t launch_step_tb2_f32(const void* src, void* dst, const Geometry& g,
                                const StepConst<F2>& k, const AxisCoef<float>* tx,
                                const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                                int pdl);
cudaError_t launch_step_tb2_f16(const void* src, void* dst, const Geometry& g,
                                const StepConst<F2>& k, const AxisCoef<float>* tx,
                                const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                                int pdl);
cudaError_t launch_step_tb2_bf16(const void* src, void* dst, const Geometry& g,
                                 const StepConst<F2>& k, const AxisCoef<float>* tx,
                                 const AxisCoef<float>* ty, int variant, int bc, cudaStream_t st,
                                 int pdl);

// Two steps per launch with the tile's input staged by TMA (FP32, Dirichlet):
// src_map describes the buffer holding time t (extent nx x ny x 9 planes,
// box 72 x 20 x 9 floats); a persistent grid of `grid` CTAs; *err is set when
// a copy did not complete within the bounded wait of `polls` mbarrier polls
// (< 0: the default bound).
cudaError_t launch_step_tb2_tma_f32(const CUtensorMap& src_map, void* dst, const Geometry& g,
                                   const StepConst<F2>& k, const AxisCoef<float>* tx,
                                   const AxisCoef<float>* ty, int variant, int grid, int* err,
                                   cudaStream_t st, int pdl, int polls);
// The same for FP16 / BF16 deviation storage (80 x 20 x 9 box of 16-bit elements).
cudaError_t launch_step_tb2_tma_f16(const CUtensorMap& src_map, void* dst, const Geometry& g,
                                    const StepConst<F2>& k, const AxisCoef<float>* tx,
                                    const AxisCoef<float>* ty, int variant, int grid, int* err,
                                    cudaStream_t st, int pdl, int polls);
cudaError_t launch_step_tb2_tma_bf16(const CUtensorMap& src_map, void* dst, const Geometry& g,
                                     const StepConst<F2>& k, const AxisCoef<float>* tx,
                                     const AxisCoef<float>* ty, int variant, int grid, int* err,
                                     cudaStream_t st, int pdl, int polls);
// Shared-memory attributes of the TMA kernels; per_sm receives CTAs per SM.
cudaError_t prepare_step_tb2_tma_f32(int* per_sm);
cudaError_t prepare_step_tb2_tma_f16(int* per_sm);
cudaError_t prepare_step_tb2_tma_bf16(int* per_sm);
// The tensor map of one population buffer for the TMA kernel (elem = 4: FP32;
// 2: FP16, or BF16 when bf16); false when the driver cannot encode it.
bool encode_tma_map(CUtensorMap* map, void* base, const Geometry& g, int elem, bool bf16);
bool encode_tma_map_f32(CUtensorMap* map, void* base, const Geometry& g);

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
// Fields of the current time (device outputs, any may be null).  ls: the
// line source (channel boundary, with t_off = the current time), else unused.
cudaError_t launch_moments(int storage, const void* src, const Geometry& g, const BaseState& b,
                           int bc, double* rho_dev, double* ux, double* uy, cudaStream_t st,
                           const LineSource& ls);
// Diagnostics: first pass writes `blocks` partial sums of kDiag doubles to
// partial[], second pass reduces them in a fixed order into out[kDiag].
constexpr int kDiag = 6;
constexpr int kDiagBlocks = 608;  // 4 per SM on a 152-SM GB300
cudaError_t launch_diagnostics(int storage, const void* src, const Geometry& g,
                               const BaseState& b, int bc, int x0, int y0, int x1, int y1,
                               double* partial, double* out, cudaStream_t st,
                               const LineSource& ls);

// Bytes per stored population.
inline size_t storage_bytes(int storage) {
    return storage == kF64 ? 8 : storage == kF32 ? 4 : 2;
}

}  // namespace lbm
