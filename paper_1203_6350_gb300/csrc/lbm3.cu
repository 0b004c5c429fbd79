// Three-dimensional scheme: D3Q15 MRT (App. A.2) with the absorbing-layer
// damping terms of Secs. 2.2.1-2.2.3, one time step per launch.
//
// Storage as in 2-D: two buffers of 15 SoA planes of deviations
// g_i = f_i - f^eq_i(rho0, u0) (FP64 or FP32), each plane nz x ny rows of
// `pitch` elements (nx rounded up to 128 bytes).  A buffer holds the
// post-collision state; a step pulls g_i(x - c_i) (zero deviation from
// outside the lattice under the Dirichlet rule, the wrapped cell when
// periodic), collides in moment space and stores at x.
//
// Collision on deviation moments m = M g (M of App. A.2, rows rho, j, e,
// epsilon, q, 3p_xx, p_ww, p_xy, p_yz, p_xz, m_xyz):
//   m += S (dm^eq(rho*, j*) - m) + damping term,
// where dm^eq = m^eq(rho, j) - m^eq(rho0, j0) of the second-order
// equilibrium, whose moments are rho, j, e = -rho + tr P, eps = rho - 5 tr P,
// q = -7/3 j, 3p_xx = 3P_xx - tr P, p_ww = P_yy - P_zz, p_ab = P_ab, m_xyz = 0
// with P = j j / rho.  The deviation of P is formed without cancellation:
//   P(rho, j) - P(rho0, j0) = (u0 j'^T + j' u0^T + j' j'^T / rho0 - u0 u0^T rho') rho0 / rho.
// The linear equilibrium has moments rho, j, -rho, rho, -7/3 j and zeros.
// Back-transform g = M^T D^-1 m (M's rows are orthogonal, D = diag(M M^T)).
// Both transforms run as butterflies over the axis pairs and the diagonals.
#include <type_traits>
#include <cmath>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_host.h"

namespace {

constexpr int kQ = 15;

// Velocity c_i in the column order of App. A.2: rest, +-x, +-y, +-z, then the
// eight diagonals (+-1, +-1, +-1) with x flipping fastest.
__host__ __device__ constexpr int d3cx(int i) {
    return i == 1 ? 1 : i == 2 ? -1 : i < 7 ? 0 : ((i - 7) & 1 ? -1 : 1);
}
__host__ __device__ constexpr int d3cy(int i) {
    return i == 3 ? 1 : i == 4 ? -1 : i < 7 ? 0 : ((i - 7) & 2 ? -1 : 1);
}
__host__ __device__ constexpr int d3cz(int i) {
    return i == 5 ? 1 : i == 6 ? -1 : i < 7 ? 0 : ((i - 7) & 4 ? -1 : 1);
}

// Row r of M at column i, as a polynomial of c_i.
__host__ __device__ constexpr int d3m(int r, int i) {
    const int x = d3cx(i), y = d3cy(i), z = d3cz(i), c2 = x * x + y * y + z * z;
    switch (r) {
        case 0: return 1;
        case 1: return x;
        case 2: return y;
        case 3: return z;
        case 4: return c2 - 2;
        case 5: return c2 == 0 ? 16 : (c2 == 1 ? -4 : 1);
        case 6: return x * (c2 == 1 ? -4 : 1);
        case 7: return y * (c2 == 1 ? -4 : 1);
        case 8: return z * (c2 == 1 ? -4 : 1);
        case 9: return 3 * x * x - c2;
        case 10: return y * y - z * z;
        case 11: return x * y;
        case 12: return y * z;
        case 13: return x * z;
        default: return x * y * z;
    }
}

// D_r = sum_i M_ri^2.
__host__ __device__ constexpr int d3norm(int r) {
    int s = 0;
    for (int i = 0; i < kQ; ++i) s += d3m(r, i) * d3m(r, i);
    return s;
}

// Host-built constants of one lattice.
template <typename CT>
struct D3Const {
    CT s[kQ];          // rates in the row order of M
    CT n, m;           // Guo weights
    CT rho0;           // far field
    CT u0[3];
    CT drf, djf[3];    // rho_f - rho0, j_f - j0
    CT dmf[kQ];        // m^eq(rho_f, j_f) - m^eq(rho0, j0)
    CT dmlf[kQ];       // the same for the linear equilibrium
};

struct D3Geom {
    int nx, ny, nz, pitch;
    unsigned plane;     // elements per population plane (< 2^31)
};

// dm^eq at (rho0 + rp, j0 + jp).  eq: second-order equilibrium.
template <typename CT>
__device__ __forceinline__ void deq2(CT rp, const CT (&jp)[3], const D3Const<CT>& k,
                                     CT (&out)[kQ]) {
    const CT ratio = k.rho0 / (k.rho0 + rp);
    const CT irho0 = CT(1) / k.rho0;
    CT P[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b)
            P[a][b] = (k.u0[a] * jp[b] + k.u0[b] * jp[a] + jp[a] * jp[b] * irho0 -
                       k.u0[a] * k.u0[b] * rp) *
                      ratio;
    const CT tr = P[0][0] + P[1][1] + P[2][2];
    out[0] = rp;
    out[1] = jp[0];
    out[2] = jp[1];
    out[3] = jp[2];
    out[4] = tr - rp;
    out[5] = rp - CT(5) * tr;
    out[6] = CT(-7.0 / 3.0) * jp[0];
    out[7] = CT(-7.0 / 3.0) * jp[1];
    out[8] = CT(-7.0 / 3.0) * jp[2];
    out[9] = CT(3) * P[0][0] - tr;
    out[10] = P[1][1] - P[2][2];
    out[11] = P[0][1];
    out[12] = P[1][2];
    out[13] = P[0][2];
    out[14] = CT(0);
}

// m = M g by butterflies: the axis pairs (+-x, +-y, +-z) and the eight
// diagonals, whose signed sums give every diagonal moment in 24 additions.
template <typename CT>
__device__ __forceinline__ void d3_forward(const CT (&g)[kQ], CT (&m)[kQ]) {
    const CT p1 = g[7] + g[8], m1 = g[7] - g[8], p2 = g[9] + g[10], m2 = g[9] - g[10];
    const CT p3 = g[11] + g[12], m3 = g[11] - g[12], p4 = g[13] + g[14], m4 = g[13] - g[14];
    const CT q1 = p1 + p2, q2 = p1 - p2, q3 = p3 + p4, q4 = p3 - p4;
    const CT r1 = m1 + m2, r2 = m1 - m2, r3 = m3 + m4, r4 = m3 - m4;
    const CT S = q1 + q3, Dz = q1 - q3, Dy = q2 + q4, Dyz = q2 - q4;
    const CT Dx = r1 + r3, Dxz = r1 - r3, Dxy = r2 + r4, Dxyz = r2 - r4;
    const CT ax = g[1] + g[2], bx = g[1] - g[2], ay = g[3] + g[4], by = g[3] - g[4];
    const CT az = g[5] + g[6], bz = g[5] - g[6];
    const CT A = ax + ay + az;
    m[0] = g[0] + A + S;
    m[1] = bx + Dx;
    m[2] = by + Dy;
    m[3] = bz + Dz;
    m[4] = S - A - CT(2) * g[0];
    m[5] = S - CT(4) * A + CT(16) * g[0];
    m[6] = Dx - CT(4) * bx;
    m[7] = Dy - CT(4) * by;
    m[8] = Dz - CT(4) * bz;
    m[9] = CT(2) * ax - ay - az;
    m[10] = ay - az;
    m[11] = Dxy;
    m[12] = Dyz;
    m[13] = Dxz;
    m[14] = Dxyz;
}

// g = M^T ph (ph = D^-1 m), the transpose of the butterflies above.
template <typename CT>
__device__ __forceinline__ void d3_backward(const CT (&ph)[kQ], CT (&g)[kQ]) {
    g[0] = ph[0] - CT(2) * ph[4] + CT(16) * ph[5];
    const CT base = ph[0] - ph[4] - CT(4) * ph[5];
    const CT X = base + CT(2) * ph[9], Y = base - ph[9] + ph[10], Z = base - ph[9] - ph[10];
    const CT vx = ph[1] - CT(4) * ph[6], vy = ph[2] - CT(4) * ph[7], vz = ph[3] - CT(4) * ph[8];
    g[1] = X + vx;
    g[2] = X - vx;
    g[3] = Y + vy;
    g[4] = Y - vy;
    g[5] = Z + vz;
    g[6] = Z - vz;
    const CT D0 = ph[0] + ph[4] + ph[5];
    const CT Ux = ph[1] + ph[6], Uy = ph[2] + ph[7], Uz = ph[3] + ph[8];
    const CT t1 = D0 + ph[12], t2 = D0 - ph[12], u1 = Uy + Uz, u2 = Uy - Uz;
    const CT cpp = t1 + u1, cmm = t1 - u1, cpm = t2 + u2, cmp = t2 - u2;  // (c_y, c_z) signs
    const CT v1 = Ux + ph[14], v2 = Ux - ph[14], w1 = ph[11] + ph[13], w2 = ph[11] - ph[13];
    const CT dpp = v1 + w1, dmm = v1 - w1, dpm = v2 + w2, dmp = v2 - w2;
    g[7] = cpp + dpp;
    g[8] = cpp - dpp;
    g[9] = cmp + dmp;
    g[10] = cmp - dmp;
    g[11] = cpm + dpm;
    g[12] = cpm - dpm;
    g[13] = cmm + dmm;
    g[14] = cmm - dmm;
}

// Collide the deviations g of one cell in place.
template <typename CT, int VAR>
__device__ __forceinline__ void d3_collide(CT (&g)[kQ], CT chi, const D3Const<CT>& k) {
    CT m[kQ];
    d3_forward(g, m);
    // rho*, j* (Guo weights, solved exactly); chi = 0 leaves rho, j
    CT rs = m[0];
    CT js[3] = {m[1], m[2], m[3]};
    if (VAR != LBM_SPONGE_NONE && chi != CT(0)) {
        const CT a = CT(1) / (CT(1) + k.n * chi), b = CT(1) / (CT(1) + k.m * chi);
        rs = (m[0] + k.n * chi * k.drf) * a;
#pragma unroll
        for (int c = 0; c < 3; ++c) js[c] = (m[1 + c] + k.m * chi * k.djf[c]) * b;
    }
    CT eq[kQ];
    deq2(rs, js, k, eq);
    CT post[kQ];
#pragma unroll
    for (int r = 0; r < kQ; ++r) post[r] = m[r] + k.s[r] * (eq[r] - m[r]);
    if (VAR == LBM_SPONGE_I) {
#pragma unroll
        for (int r = 0; r < kQ; ++r) post[r] += chi * (k.dmf[r] - m[r]);
    } else if (VAR == LBM_SPONGE_II) {
#pragma unroll
        for (int r = 0; r < kQ; ++r) post[r] += chi * (k.dmf[r] - eq[r]);
    } else if (VAR == LBM_SPONGE_III) {
        const CT lin[kQ] = {rs, js[0], js[1], js[2], -rs, rs, CT(-7.0 / 3.0) * js[0],
                            CT(-7.0 / 3.0) * js[1], CT(-7.0 / 3.0) * js[2], CT(0), CT(0),
                            CT(0), CT(0), CT(0), CT(0)};
#pragma unroll
        for (int r = 0; r < kQ; ++r) post[r] += chi * (k.dmlf[r] - lin[r]);
    }
    // rows 0-3 (rho', j'): a correctly rounded 1/D, since 15 fl(1/15) and
    // 10 fl(1/10) differ from 1 by 5.2e-8 and 1.5e-8 in FP32 and would scale the
    // conserved deviations by that every step (the residual is 0 in FP64)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        constexpr bool f32 = std::is_same<CT, float>::value;
        const CT lo = CT(f32 ? 1.0 / d3norm(r) - double(float(1.0 / d3norm(r))) : 0.0);
        post[r] = fma(post[r], CT(1.0 / d3norm(r)), post[r] * lo);
    }
#pragma unroll
    for (int r = 4; r < kQ; ++r) post[r] *= CT(1.0 / d3norm(r));
    d3_backward(post, g);
}

__device__ __forceinline__ int wrap(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

constexpr int kBX = 64, kBY = 4;

// Element offset of plane i, position o: 32-bit when all 15 planes stay below
// 2^32 elements (NARROW), else 64-bit.
template <bool NARROW>
__device__ __forceinline__ size_t plane_off(int i, unsigned plane, unsigned o) {
    if (NARROW) return static_cast<unsigned>(i) * plane + o;
    return static_cast<size_t>(i) * plane + o;
}

template <typename T, int VAR, int BC, bool NARROW>
__global__ void __launch_bounds__(kBX * kBY)
    d3_step_kernel(const T* __restrict__ src, T* __restrict__ dst, D3Geom g, D3Const<T> k,
                   const T* __restrict__ chix, const T* __restrict__ chiy,
                   const T* __restrict__ chiz) {
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y = blockIdx.y * kBY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const unsigned row = static_cast<unsigned>(g.pitch);
    const unsigned slab = row * static_cast<unsigned>(g.ny);
    const unsigned o = (static_cast<unsigned>(z) * g.ny + y) * row + x;
    T f[kQ];
    if (x > 0 && x + 1 < g.nx && y > 0 && y + 1 < g.ny && z > 0 && z + 1 < g.nz) {
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const int d = d3cx(i) + d3cy(i) * static_cast<int>(row) +
                          d3cz(i) * static_cast<int>(slab);
            f[i] = src[plane_off<NARROW>(i, g.plane, o - d)];
        }
    } else {
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            int sx = x - d3cx(i), sy = y - d3cy(i), sz = z - d3cz(i);
            if (BC == LBM_BC_PERIODIC) {
                sx = wrap(sx, g.nx);
                sy = wrap(sy, g.ny);
                sz = wrap(sz, g.nz);
            } else if (sx < 0 || sx >= g.nx || sy < 0 || sy >= g.ny || sz < 0 || sz >= g.nz) {
                f[i] = T(0);
                continue;
            }
            f[i] = src[plane_off<NARROW>(i, g.plane,
                                         (static_cast<unsigned>(sz) * g.ny + sy) * row + sx)];
        }
    }
    T chi = T(0);
    if (VAR != LBM_SPONGE_NONE) chi = fmax(fmax(chix[x], chiy[y]), chiz[z]);
    d3_collide<T, VAR>(f, chi, k);
#pragma unroll
    for (int i = 0; i < kQ; ++i) dst[plane_off<NARROW>(i, g.plane, o)] = f[i];
}

// Slot x of plane i <- f^eq_i(rho, u at x + c_i) - f^eq_i(rho0, u0) (the
// wrapped cell when periodic; 0 when x + c_i is outside, a slot no pull reads).
// Fields are FP64 [nz][ny][nx] on the device.
template <typename T>
__global__ void d3_init_kernel(T* __restrict__ dst, D3Geom g, double rho0, double ux0,
                               double uy0, double uz0, int bc, const double* __restrict__ rho,
                               const double* __restrict__ ux, const double* __restrict__ uy,
                               const double* __restrict__ uz) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx) return;
    const double w[3] = {2.0 / 9.0, 1.0 / 9.0, 1.0 / 72.0};
    const double u0[3] = {ux0, uy0, uz0};
    const unsigned o = (static_cast<unsigned>(z) * g.ny + y) * g.pitch + x;
    for (int i = 0; i < kQ; ++i) {
        int sx = x + d3cx(i), sy = y + d3cy(i), sz = z + d3cz(i);
        double v = 0.0;
        if (bc == LBM_BC_PERIODIC) {
            sx = wrap(sx, g.nx);
            sy = wrap(sy, g.ny);
            sz = wrap(sz, g.nz);
        }
        if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz) {
            const size_t c = (static_cast<size_t>(sz) * g.ny + sy) * g.nx + sx;
            const double r = rho[c], u[3] = {ux[c], uy[c], uz[c]};
            const int ci[3] = {d3cx(i), d3cy(i), d3cz(i)};
            // f^eq(rho, u) - f^eq(rho0, u0) over w_i, term by term
            double cu = 0, cu0 = 0, uu = 0, uu0 = 0;
            for (int a = 0; a < 3; ++a) {
                cu += ci[a] * u[a];
                cu0 += ci[a] * u0[a];
                uu += u[a] * u[a];
                uu0 += u0[a] * u0[a];
            }
            const double dr = r - rho0;
            const double dlin = dr + 3.0 * (r * cu - rho0 * cu0);
            const double dquad = 4.5 * (r * cu * cu - rho0 * cu0 * cu0) - 1.5 * (r * uu - rho0 * uu0);
            v = w[i == 0 ? 0 : (i < 7 ? 1 : 2)] * (dlin + dquad);
        }
        dst[static_cast<size_t>(i) * g.plane + o] = static_cast<T>(v);
    }
}

// Deviations (rho', j - rho0 u0) of the pulled (pre-collision) state at a cell.
template <typename T>
__device__ __forceinline__ void d3_pulled_moments(const T* __restrict__ src, const D3Geom& g,
                                                  int bc, int x, int y, int z, double (&m)[4]) {
    m[0] = m[1] = m[2] = m[3] = 0.0;
    for (int i = 0; i < kQ; ++i) {
        int sx = x - d3cx(i), sy = y - d3cy(i), sz = z - d3cz(i);
        double v = 0.0;
        if (bc == LBM_BC_PERIODIC) {
            sx = wrap(sx, g.nx);
            sy = wrap(sy, g.ny);
            sz = wrap(sz, g.nz);
        }
        if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz)
            v = static_cast<double>(src[static_cast<size_t>(i) * g.plane +
                                        (static_cast<unsigned>(sz) * g.ny + sy) * g.pitch + sx]);
        m[0] += v;
        m[1] += d3cx(i) * v;
        m[2] += d3cy(i) * v;
        m[3] += d3cz(i) * v;
    }
}

// rho' and u of the pulled (pre-collision) state, FP64 [nz][ny][nx].
template <typename T>
__global__ void d3_moments_kernel(const T* __restrict__ src, D3Geom g, double rho0, double ux0,
                                  double uy0, double uz0, int bc, double* __restrict__ rho,
                                  double* __restrict__ ux, double* __restrict__ uy,
                                  double* __restrict__ uz) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx) return;
    double m[4];
    d3_pulled_moments(src, g, bc, x, y, z, m);
    // deviations of rho and j from the base f^eq(rho0, u0), whose moments are rho0, rho0 u0
    const double r = rho0 + m[0];
    const size_t c = (static_cast<size_t>(z) * g.ny + y) * g.nx + x;
    rho[c] = m[0];
    ux[c] = (rho0 * ux0 + m[1]) / r;
    uy[c] = (rho0 * uy0 + m[2]) / r;
    uz[c] = (rho0 * uz0 + m[3]) / r;
}

constexpr int kD3Diag = 7;           // sums of lbm3_diagnostics
constexpr int kD3DiagThreads = 256;
constexpr int kD3DiagBlocks = 608;   // fixed, so that the summation order is fixed

__device__ __forceinline__ double d3_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// First pass: thread t of block b takes the region's cells b * 256 + t,
// + 608 * 256, ... in x-fastest order and writes the block's kD3Diag sums to
// partial[b].
template <typename T>
__global__ void __launch_bounds__(kD3DiagThreads)
    d3_diag_partial_kernel(const T* __restrict__ src, D3Geom g, int bc, double rho0, double ux0,
                           double uy0, double uz0, int x0, int y0, int z0, int wx, int wy,
                           long long ncell, double* __restrict__ partial) {
    double acc[kD3Diag] = {0, 0, 0, 0, 0, 0, 0};
    const double u0[3] = {ux0, uy0, uz0};
    for (long long c = static_cast<long long>(blockIdx.x) * kD3DiagThreads + threadIdx.x;
         c < ncell; c += static_cast<long long>(gridDim.x) * kD3DiagThreads) {
        const int x = x0 + static_cast<int>(c % wx);
        const int y = y0 + static_cast<int>((c / wx) % wy);
        const int z = z0 + static_cast<int>(c / (static_cast<long long>(wx) * wy));
        double m[4];
        d3_pulled_moments(src, g, bc, x, y, z, m);
        // u - u0 = (j' - rho' u0) / rho
        const double inv = 1.0 / (rho0 + m[0]);
        double du2 = 0.0;
        bool finite = isfinite(m[0]);
        for (int a = 0; a < 3; ++a) {
            const double du = (m[1 + a] - m[0] * u0[a]) * inv;
            du2 += du * du;
            finite = finite && isfinite(du);
        }
        acc[0] += m[0];
        acc[1] += m[1];
        acc[2] += m[2];
        acc[3] += m[3];
        acc[4] += m[0] * m[0] / (6.0 * rho0) + 0.5 * rho0 * du2;  // c_s^2 = 1/3
        acc[5] += m[0] * m[0];
        acc[6] += finite ? 0.0 : 1.0;
    }
    __shared__ double red[kD3Diag][kD3DiagThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kD3Diag; ++q) {
        const double v = d3_warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kD3Diag) {
        double s = 0.0;
        for (int k = 0; k < kD3DiagThreads / 32; ++k) s += red[threadIdx.x][k];
        partial[blockIdx.x * kD3Diag + threadIdx.x] = s;
    }
}

// Second pass: one block adds the partials in a fixed order.
__global__ void __launch_bounds__(kD3DiagThreads)
    d3_diag_final_kernel(const double* __restrict__ partial, double* __restrict__ out) {
    __shared__ double red[kD3Diag][kD3DiagThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kD3Diag; ++q) {
        double s = 0.0;
        for (int k = threadIdx.x; k < kD3DiagBlocks; k += kD3DiagThreads)
            s += partial[k * kD3Diag + q];
        s = d3_warp_sum(s);
        if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < kD3Diag) {
        double s = 0.0;
        for (int k = 0; k < kD3DiagThreads / 32; ++k) s += red[threadIdx.x][k];
        out[threadIdx.x] = s;
    }
}

}  // namespace

struct lbm3_ctx {
    int nx = 0, ny = 0, nz = 0;
    int storage = LBM_F32, bc = LBM_BC_DIRICHLET_EQ, variant = LBM_SPONGE_NONE;
    D3Geom g{};
    double rho0 = 1, u0[3] = {0, 0, 0};
    double s[kQ] = {};
    double n = 0.5, m = 0.5;
    double rho_f = 1, u_f[3] = {0, 0, 0};
    void* buf[2] = {nullptr, nullptr};
    void* chi[3] = {nullptr, nullptr, nullptr};
    int cur = 0;
    bool ready = false;
    long long time = 0;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_lbm3_error;

int fail3(lbm3_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    g_lbm3_error = msg;
    return code;
}

size_t elem_size(int storage) { return storage == LBM_F64 ? 8 : 4; }

template <typename CT>
D3Const<CT> make_const(const lbm3_ctx& h) {
    D3Const<CT> k{};
    for (int r = 0; r < kQ; ++r) k.s[r] = static_cast<CT>(h.s[r]);
    k.n = static_cast<CT>(h.n);
    k.m = static_cast<CT>(h.m);
    k.rho0 = static_cast<CT>(h.rho0);
    const double j0[3] = {h.rho0 * h.u0[0], h.rho0 * h.u0[1], h.rho0 * h.u0[2]};
    const double jf[3] = {h.rho_f * h.u_f[0], h.rho_f * h.u_f[1], h.rho_f * h.u_f[2]};
    double djf[3], P[3][3], P0[3][3];
    for (int a = 0; a < 3; ++a) {
        k.u0[a] = static_cast<CT>(h.u0[a]);
        djf[a] = jf[a] - j0[a];
        k.djf[a] = static_cast<CT>(djf[a]);
        for (int b = 0; b < 3; ++b) {
            P[a][b] = jf[a] * jf[b] / h.rho_f;
            P0[a][b] = j0[a] * j0[b] / h.rho0;
        }
    }
    const double drf = h.rho_f - h.rho0;
    k.drf = static_cast<CT>(drf);
    double dP[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) dP[a][b] = P[a][b] - P0[a][b];
    const double tr = dP[0][0] + dP[1][1] + dP[2][2];
    const double eq[kQ] = {drf,        djf[0],         djf[1],         djf[2],
                           tr - drf,   drf - 5 * tr,   -7.0 / 3 * djf[0], -7.0 / 3 * djf[1],
                           -7.0 / 3 * djf[2], 3 * dP[0][0] - tr, dP[1][1] - dP[2][2], dP[0][1],
                           dP[1][2],   dP[0][2],       0.0};
    const double lin[kQ] = {drf, djf[0], djf[1], djf[2], -drf, drf, -7.0 / 3 * djf[0],
                            -7.0 / 3 * djf[1], -7.0 / 3 * djf[2], 0, 0, 0, 0, 0, 0};
    for (int r = 0; r < kQ; ++r) {
        k.dmf[r] = static_cast<CT>(eq[r]);
        k.dmlf[r] = static_cast<CT>(lin[r]);
    }
    return k;
}

template <typename T>
cudaError_t launch_step(lbm3_ctx* h) {
    const dim3 block(kBX, kBY);
    const dim3 grid((h->nx + kBX - 1) / kBX, (h->ny + kBY - 1) / kBY, h->nz);
    const T* s = static_cast<const T*>(h->buf[h->cur]);
    T* d = static_cast<T*>(h->buf[h->cur ^ 1]);
    const D3Const<T> k = make_const<T>(*h);
    const T* cx = static_cast<const T*>(h->chi[0]);
    const T* cy = static_cast<const T*>(h->chi[1]);
    const T* cz = static_cast<const T*>(h->chi[2]);
    const bool narrow = static_cast<unsigned long long>(kQ) * h->g.plane < (1ull << 32);
#define LBM3_CASE(V, B)                                                                          \
    if (h->variant == V && h->bc == B) {                                                         \
        if (narrow)                                                                              \
            d3_step_kernel<T, V, B, true><<<grid, block, 0, h->stream>>>(s, d, h->g, k, cx, cy, \
                                                                          cz);                   \
        else                                                                                     \
            d3_step_kernel<T, V, B, false><<<grid, block, 0, h->stream>>>(s, d, h->g, k, cx, cy, \
                                                                           cz);                  \
        return cudaGetLastError();                                                               \
    }
    LBM3_CASE(LBM_SPONGE_NONE, LBM_BC_DIRICHLET_EQ)
    LBM3_CASE(LBM_SPONGE_I, LBM_BC_DIRICHLET_EQ)
    LBM3_CASE(LBM_SPONGE_II, LBM_BC_DIRICHLET_EQ)
    LBM3_CASE(LBM_SPONGE_III, LBM_BC_DIRICHLET_EQ)
    LBM3_CASE(LBM_SPONGE_NONE, LBM_BC_PERIODIC)
    LBM3_CASE(LBM_SPONGE_I, LBM_BC_PERIODIC)
    LBM3_CASE(LBM_SPONGE_II, LBM_BC_PERIODIC)
    LBM3_CASE(LBM_SPONGE_III, LBM_BC_PERIODIC)
#undef LBM3_CASE
    return cudaErrorInvalidValue;
}

// Upload a host FP64 table of n values as the storage type.
int upload_table(lbm3_ctx* h, int axis, const double* v, int n) {
    if (!v) return fail3(h, LBM_ERR_ARG, "NULL chi array");
    if (h->storage == LBM_F64) {
        if (cudaMemcpyAsync(h->chi[axis], v, n * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
            return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        return cudaStreamSynchronize(h->stream) == cudaSuccess
                   ? LBM_OK
                   : fail3(h, LBM_ERR_CUDA, "stream synchronize failed");
    }
    float* tmp = new float[n];
    for (int i = 0; i < n; ++i) tmp[i] = static_cast<float>(v[i]);
    const cudaError_t e1 = cudaMemcpyAsync(h->chi[axis], tmp, n * sizeof(float),
                                           cudaMemcpyHostToDevice, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    delete[] tmp;
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return LBM_OK;
}

bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int lbm3_create(int nx, int ny, int nz, lbm_storage storage, double rho0, double ux0, double uy0,
                double uz0, const double* s, double n, double m, lbm_bc bc, void* cuda_stream,
                lbm3_handle* out) {
    if (!out) return fail3(nullptr, LBM_ERR_ARG, "NULL out");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail3(nullptr, LBM_ERR_ARG, "sizes must be >= 1");
    if (ny > 65535 || nz > 65535)
        return fail3(nullptr, LBM_ERR_ARG, "ny and nz must be <= 65535 (grid dimensions)");
    if (storage != LBM_F64 && storage != LBM_F32)
        return fail3(nullptr, LBM_ERR_ARG, "storage must be LBM_F64 or LBM_F32");
    if (bc != LBM_BC_DIRICHLET_EQ && bc != LBM_BC_PERIODIC)
        return fail3(nullptr, LBM_ERR_ARG, "bc must be LBM_BC_DIRICHLET_EQ or LBM_BC_PERIODIC");
    if (!(rho0 > 0) || !std::isfinite(rho0) || !std::isfinite(ux0) || !std::isfinite(uy0) ||
        !std::isfinite(uz0))
        return fail3(nullptr, LBM_ERR_ARG, "rho0 must be > 0 and the far field finite");
    if (!s || !finite_all(s, kQ)) return fail3(nullptr, LBM_ERR_ARG, "rates NULL or not finite");
    if (!(n >= 0) || !(m >= 0) || !std::isfinite(n) || !std::isfinite(m))
        return fail3(nullptr, LBM_ERR_ARG, "Guo weights n, m must be finite and >= 0");
    const size_t es = elem_size(storage);
    const long long pitch = ((static_cast<long long>(nx) * es + 127) / 128) * 128 / es;
    const long long plane = pitch * ny * nz;
    if (plane >= (1ll << 31)) return fail3(nullptr, LBM_ERR_ARG, "lattice too large (plane >= 2^31)");
    lbm3_ctx* h = new lbm3_ctx;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->storage = storage;
    h->bc = bc;
    h->g = D3Geom{nx, ny, nz, static_cast<int>(pitch), static_cast<unsigned>(plane)};
    h->rho0 = h->rho_f = rho0;
    h->u0[0] = h->u_f[0] = ux0;
    h->u0[1] = h->u_f[1] = uy0;
    h->u0[2] = h->u_f[2] = uz0;
    for (int r = 0; r < kQ; ++r) h->s[r] = s[r];
    h->n = n;
    h->m = m;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t bytes = static_cast<size_t>(plane) * kQ * es;
    bool ok = cudaMalloc(&h->buf[0], bytes) == cudaSuccess &&
              cudaMalloc(&h->buf[1], bytes) == cudaSuccess &&
              cudaMalloc(&h->chi[0], nx * es) == cudaSuccess &&
              cudaMalloc(&h->chi[1], ny * es) == cudaSuccess &&
              cudaMalloc(&h->chi[2], nz * es) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbm3_destroy(h);
        return fail3(nullptr, LBM_ERR_OOM, "device allocation failed");
    }
    if (cudaMemsetAsync(h->buf[0], 0, bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->buf[1], 0, bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->chi[0], 0, nx * es, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->chi[1], 0, ny * es, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->chi[2], 0, nz * es, h->stream) != cudaSuccess ||
        (lbm::canary_requested() &&
         (lbm::paint_canary(h->buf[0], es, nx, pitch, 1ll * kQ * ny * nz, h->stream) != cudaSuccess ||
          lbm::paint_canary(h->buf[1], es, nx, pitch, 1ll * kQ * ny * nz, h->stream) != cudaSuccess)) ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        lbm3_destroy(h);
        return fail3(nullptr, LBM_ERR_CUDA, "clearing the buffers failed");
    }
    *out = h;
    for (int r = 0; r < kQ; ++r)
        if (!(s[r] > 0 && s[r] < 2))
            return fail3(h, LBM_WARN_UNSTABLE_PARAMS, "a rate outside (0, 2)");
    return LBM_OK;
}

int lbm3_set_sponge(lbm3_handle h, lbm_variant variant, const double* chi_x, const double* chi_y,
                    const double* chi_z, double rho_ref, double ux_ref, double uy_ref,
                    double uz_ref) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "NULL handle");
    if (variant < LBM_SPONGE_NONE || variant > LBM_SPONGE_III)
        return fail3(h, LBM_ERR_ARG, "variant must be none, I, II or III");
    if (!(rho_ref > 0) || !std::isfinite(rho_ref) || !std::isfinite(ux_ref) ||
        !std::isfinite(uy_ref) || !std::isfinite(uz_ref))
        return fail3(h, LBM_ERR_ARG, "reference state must be finite with rho_ref > 0");
    const double* arr[3] = {chi_x, chi_y, chi_z};
    const int len[3] = {h->nx, h->ny, h->nz};
    double cmax = 0;
    for (int a = 0; a < 3; ++a) {
        if (!arr[a]) return fail3(h, LBM_ERR_ARG, "NULL chi array");
        for (int i = 0; i < len[a]; ++i) {
            if (!std::isfinite(arr[a][i]) || arr[a][i] < 0)
                return fail3(h, LBM_ERR_ARG, "chi must be finite and >= 0");
            cmax = cmax > arr[a][i] ? cmax : arr[a][i];
        }
    }
    for (int a = 0; a < 3; ++a) {
        const int rc = upload_table(h, a, arr[a], len[a]);
        if (rc != LBM_OK) return rc;
    }
    h->variant = variant;
    h->rho_f = rho_ref;
    h->u_f[0] = ux_ref;
    h->u_f[1] = uy_ref;
    h->u_f[2] = uz_ref;
    double smax = 0;
    for (int r = 4; r < kQ; ++r) smax = smax > h->s[r] ? smax : h->s[r];
    if ((variant == LBM_SPONGE_I && smax + cmax > 2) ||
        ((variant == LBM_SPONGE_II || variant == LBM_SPONGE_III) && cmax > 4 / h->s[0]))
        return fail3(h, LBM_WARN_UNSTABLE_PARAMS, "chi beyond the critical value");
    return LBM_OK;
}

int lbm3_init_equilibrium(lbm3_handle h, const double* rho, const double* ux, const double* uy,
                          const double* uz) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!rho || !ux || !uy || !uz) return fail3(h, LBM_ERR_ARG, "NULL field");
    const size_t cells = static_cast<size_t>(h->nx) * h->ny * h->nz;
    double* d = nullptr;
    if (cudaMallocAsync(&d, 4 * cells * sizeof(double), h->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail3(h, LBM_ERR_OOM, "device allocation failed");
    }
    const double* src[4] = {rho, ux, uy, uz};
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 4 && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(d + a * cells, src[a], cells * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) {
        const dim3 block(128), grid((h->nx + 127) / 128, h->ny, h->nz);
        if (h->storage == LBM_F64)
            d3_init_kernel<double><<<grid, block, 0, h->stream>>>(
                static_cast<double*>(h->buf[0]), h->g, h->rho0, h->u0[0], h->u0[1], h->u0[2],
                h->bc, d, d + cells, d + 2 * cells, d + 3 * cells);
        else
            d3_init_kernel<float><<<grid, block, 0, h->stream>>>(
                static_cast<float*>(h->buf[0]), h->g, h->rho0, h->u0[0], h->u0[1], h->u0[2],
                h->bc, d, d + cells, d + 2 * cells, d + 3 * cells);
        e = cudaGetLastError();
    }
    cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(e));
    h->cur = 0;
    h->time = 0;
    h->ready = true;
    return LBM_OK;
}

int lbm3_step(lbm3_handle h, int nsteps) {
    const lbm::NvtxRange nvtx("lbm3_step");
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "NULL handle");
    if (nsteps < 0) return fail3(h, LBM_ERR_ARG, "nsteps < 0");
    if (!h->ready) return fail3(h, LBM_ERR_STATE, "step before lbm3_init_equilibrium");
    for (int t = 0; t < nsteps; ++t) {
        const cudaError_t e = h->storage == LBM_F64 ? launch_step<double>(h) : launch_step<float>(h);
        if (e != cudaSuccess) return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(e));
        h->cur ^= 1;
        ++h->time;
    }
    return LBM_OK;
}

int lbm3_moments(lbm3_handle h, double* rho_dev, double* ux, double* uy, double* uz) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!rho_dev || !ux || !uy || !uz) return fail3(h, LBM_ERR_ARG, "NULL output");
    if (!h->ready) return fail3(h, LBM_ERR_STATE, "moments before lbm3_init_equilibrium");
    const size_t cells = static_cast<size_t>(h->nx) * h->ny * h->nz;
    double* d = nullptr;
    if (cudaMallocAsync(&d, 4 * cells * sizeof(double), h->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail3(h, LBM_ERR_OOM, "device allocation failed");
    }
    const dim3 block(128), grid((h->nx + 127) / 128, h->ny, h->nz);
    if (h->storage == LBM_F64)
        d3_moments_kernel<double><<<grid, block, 0, h->stream>>>(
            static_cast<const double*>(h->buf[h->cur]), h->g, h->rho0, h->u0[0], h->u0[1],
            h->u0[2], h->bc, d, d + cells, d + 2 * cells, d + 3 * cells);
    else
        d3_moments_kernel<float><<<grid, block, 0, h->stream>>>(
            static_cast<const float*>(h->buf[h->cur]), h->g, h->rho0, h->u0[0], h->u0[1],
            h->u0[2], h->bc, d, d + cells, d + 2 * cells, d + 3 * cells);
    cudaError_t e = cudaGetLastError();
    double* dst[4] = {rho_dev, ux, uy, uz};
    for (int a = 0; a < 4 && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(dst[a], d + a * cells, cells * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream);
    cudaFreeAsync(d, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
    return LBM_OK;
}

int lbm3_diagnostics(lbm3_handle h, int x0, int y0, int z0, int x1, int y1, int z1,
                     double out[7]) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!out) return fail3(h, LBM_ERR_ARG, "NULL out");
    if (!h->ready) return fail3(h, LBM_ERR_STATE, "diagnostics before lbm3_init_equilibrium");
    if (x0 < 0 || y0 < 0 || z0 < 0 || x1 > h->nx || y1 > h->ny || z1 > h->nz || x0 > x1 ||
        y0 > y1 || z0 > z1)
        return fail3(h, LBM_ERR_ARG, "region outside the lattice");
    const long long ncell = static_cast<long long>(x1 - x0) * (y1 - y0) * (z1 - z0);
    double* d = nullptr;
    const size_t bytes = (kD3DiagBlocks + 1) * kD3Diag * sizeof(double);
    if (cudaMallocAsync(&d, bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail3(h, LBM_ERR_OOM, "device allocation failed");
    }
    double* res = d + kD3DiagBlocks * kD3Diag;
    cudaError_t e = cudaSuccess;
    if (ncell == 0) {
        e = cudaMemsetAsync(res, 0, kD3Diag * sizeof(double), h->stream);
    } else {
        const int wx = x1 - x0, wy = y1 - y0;
        if (h->storage == LBM_F64)
            d3_diag_partial_kernel<double><<<kD3DiagBlocks, kD3DiagThreads, 0, h->stream>>>(
                static_cast<const double*>(h->buf[h->cur]), h->g, h->bc, h->rho0, h->u0[0],
                h->u0[1], h->u0[2], x0, y0, z0, wx, wy, ncell, d);
        else
            d3_diag_partial_kernel<float><<<kD3DiagBlocks, kD3DiagThreads, 0, h->stream>>>(
                static_cast<const float*>(h->buf[h->cur]), h->g, h->bc, h->rho0, h->u0[0],
                h->u0[1], h->u0[2], x0, y0, z0, wx, wy, ncell, d);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            d3_diag_final_kernel<<<1, kD3DiagThreads, 0, h->stream>>>(d, res);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, res, kD3Diag * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
    if (out[6] > 0) return fail3(h, LBM_ERR_NONFINITE, "the state holds non-finite values");
    return LBM_OK;
}

size_t lbm3_state_bytes(lbm3_handle h) {
    return h ? static_cast<size_t>(h->g.plane) * kQ * elem_size(h->storage) : 0;
}

int lbm3_get_state(lbm3_handle h, void* dst, size_t bytes, int64_t* time) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!dst || bytes != lbm3_state_bytes(h))
        return fail3(h, LBM_ERR_ARG, "dst / bytes do not match lbm3_state_bytes");
    if (!h->ready) return fail3(h, LBM_ERR_STATE, "no state before lbm3_init_equilibrium");
    cudaError_t e = cudaMemcpyAsync(dst, h->buf[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(e));
    if (time) *time = h->time;
    return LBM_OK;
}

int lbm3_set_state(lbm3_handle h, const void* src, size_t bytes, int64_t time) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!src || bytes != lbm3_state_bytes(h))
        return fail3(h, LBM_ERR_ARG, "src / bytes do not match lbm3_state_bytes");
    if (time < 0) return fail3(h, LBM_ERR_ARG, "time < 0");
    cudaError_t e = cudaMemcpyAsync(h->buf[0], src, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail3(h, LBM_ERR_CUDA, cudaGetErrorString(e));
    h->cur = 0;
    h->time = time;
    h->ready = true;
    return LBM_OK;
}

int64_t lbm3_time(lbm3_handle h) { return h ? h->time : -1; }

void lbm3_destroy(lbm3_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->buf)
        if (p) cudaFree(p);
    for (void* p : h->chi)
        if (p) cudaFree(p);
    delete h;
}

const char* lbm3_last_error(lbm3_handle h) { return h ? h->err.c_str() : g_lbm3_error.c_str(); }

}  // extern "C"
