// Per-cell arithmetic of the D2Q9 MRT step with absorbing terms, in moment
// space on population deviations.  Device code only.
//
// The scheme is Eq. (blbs-abc-1) of Xu & Sagaut (arXiv:1203.6350) with
// Gamma = chi I (Eq. eq:gamma) and Lambda = M^-1 S M (Sec. 2.1), for the three
// damping terms of Secs. 2.2.1-2.2.3.  Because Gamma = chi I commutes with M,
// the whole collision is done on the nine moments m = M g:
//
//   m_k^+ = m_k + s_k (m_k^eq(rho*, j*) - m_k) + chi T_k,
//     type I   T_k = m_k^eq(q_ref) - m_k
//     type II  T_k = m_k^eq(q_ref) - m_k^eq(rho*, j*)
//     type III T_k = m_k^Leq(q_ref) - m_k^Leq(rho*, j*)
//
// and g^+ = M^-1 m^+ = M^T D^-1 m^+ with D = M M^T = diag(9,6,6,36,36,12,12,4,4).
// The moment equilibria of f^eq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
// are (rho, j_x, j_y, -2 rho + 3|j|^2/rho, rho - 3|j|^2/rho, -j_x, -j_y,
// (j_x^2 - j_y^2)/rho, j_x j_y/rho); those of its linear part w_i (rho + 3 c.j)
// drop the |j|^2 / rho terms and the last two rows.
//
// Populations are deviations g = f - f^eq(rho0, u0) so that single precision
// keeps the ~1e-3 acoustic signal: every quantity below is a deviation from
// the base state, and the quadratic equilibria are differenced in a form that
// never subtracts two O(1) numbers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {

// Velocity set in the order of the rows 1-2 of M (App. A.1).
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}

// 16-bit storage keeps q_i = g_i * 2^e_i: a power of two per plane that puts
// g_i / w_i (w = 4/9, 1/9, 1/36) near the middle of the format's range and is
// exact to apply.
__host__ __device__ constexpr int scale_exp(int i) { return 8 + (i == 0 ? 1 : i < 5 ? 3 : 5); }
__host__ __device__ constexpr float pow2f(int e) {
    float r = 1.0f;
    for (int k = 0; k < (e < 0 ? -e : e); ++k) r = e < 0 ? r * 0.5f : r * 2.0f;
    return r;
}

template <typename T>
struct Codec;
template <>
struct Codec<double> {
    using CT = double;
    template <int I>
    __device__ static __forceinline__ double dec(double v) { return v; }
    template <int I>
    __device__ static __forceinline__ double enc(double v) { return v; }
};
template <>
struct Codec<float> {
    using CT = float;
    template <int I>
    __device__ static __forceinline__ float dec(float v) { return v; }
    template <int I>
    __device__ static __forceinline__ float enc(float v) { return v; }
};
template <>
struct Codec<__half> {
    using CT = float;
    template <int I>
    __device__ static __forceinline__ float dec(__half v) {
        return __half2float(v) * pow2f(-scale_exp(I));
    }
    template <int I>
    __device__ static __forceinline__ __half enc(float v) {
        return __float2half_rn(v * pow2f(scale_exp(I)));
    }
};
template <>
struct Codec<__nv_bfloat16> {
    using CT = float;
    template <int I>
    __device__ static __forceinline__ float dec(__nv_bfloat16 v) {
        return __bfloat162float(v) * pow2f(-scale_exp(I));
    }
    template <int I>
    __device__ static __forceinline__ __nv_bfloat16 enc(float v) {
        return __float2bfloat16_rn(v * pow2f(scale_exp(I)));
    }
};

__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// Collide one cell in place: g holds the nine pulled deviations on entry and
// the post-collision deviations on exit.  chi is the absorbing strength here.
template <typename CT, int VAR>
__device__ __forceinline__ void collide(CT (&g)[9], CT chi, const StepConst<CT>& k) {
    // m = M g (App. A.1), written as sums and differences
    const CT a13 = g[1] - g[3], a24 = g[2] - g[4];
    const CT b57 = g[5] - g[7], c86 = g[8] - g[6];
    const CT s14 = (g[1] + g[3]) + (g[2] + g[4]);
    const CT s58 = (g[5] + g[7]) + (g[6] + g[8]);
    CT m[9];
    m[0] = g[0] + s14 + s58;                          // rho'
    m[1] = a13 + b57 + c86;                           // j_x'
    m[2] = a24 + b57 - c86;                           // j_y'
    m[3] = CT(-4) * g[0] - s14 + CT(2) * s58;         // e
    m[4] = CT(4) * g[0] - CT(2) * s14 + s58;          // epsilon
    m[5] = CT(-2) * a13 + b57 + c86;                  // q_x
    m[6] = CT(-2) * a24 + b57 - c86;                  // q_y
    m[7] = (g[1] + g[3]) - (g[2] + g[4]);             // p_xx
    m[8] = (g[5] + g[7]) - (g[6] + g[8]);             // p_xy

    // rho*, j*: the Guo definitions solved exactly (sum F = chi (rho_f - rho*),
    // sum c F = chi (j_f - j*)), as deviations from the base state.
    const CT rn = rcp(CT(1) + k.n * chi);
    const CT rm = rcp(CT(1) + k.m * chi);
    const CT drs = (m[0] + k.n * chi * k.drf) * rn;
    const CT djxs = (m[1] + k.m * chi * k.djfx) * rm;
    const CT djys = (m[2] + k.m * chi * k.djfy) * rm;

    // m^eq(rho*, j*) - m^eq(rho0, j0) without cancellation:
    //   |j*|^2/rho* - |j0|^2/rho0 = (rho0 (|j*|^2 - |j0|^2) - |j0|^2 drho*) / (rho* rho0)
    const CT inv = rcp((k.rho0 + drs) * k.rho0);
    const CT ax = djxs * (CT(2) * k.jx0 + djxs);
    const CT ay = djys * (CT(2) * k.jy0 + djys);
    const CT q = (k.rho0 * (ax + ay) - k.jj0 * drs) * inv;
    const CT pxx = (k.rho0 * (ax - ay) - k.jxy0 * drs) * inv;
    const CT pxy = (k.rho0 * (djxs * k.jy0 + k.jx0 * djys + djxs * djys) - k.pxy0 * drs) * inv;
    CT meq[9];
    meq[0] = drs;
    meq[1] = djxs;
    meq[2] = djys;
    meq[3] = CT(-2) * drs + CT(3) * q;
    meq[4] = drs - CT(3) * q;
    meq[5] = -djxs;
    meq[6] = -djys;
    meq[7] = pxx;
    meq[8] = pxy;

    CT t[9];
    if (VAR == kTypeI) {
#pragma unroll
        for (int i = 0; i < 9; ++i) t[i] = k.dmeq_ref[i] - m[i];
    } else if (VAR == kTypeII) {
#pragma unroll
        for (int i = 0; i < 9; ++i) t[i] = k.dmeq_ref[i] - meq[i];
    } else if (VAR == kTypeIII) {
        const CT dr = k.drf - drs, dx = k.djfx - djxs, dy = k.djfy - djys;
        t[0] = dr;
        t[1] = dx;
        t[2] = dy;
        t[3] = CT(-2) * dr;
        t[4] = dr;
        t[5] = -dx;
        t[6] = -dy;
        t[7] = CT(0);
        t[8] = CT(0);
    }

    // relax and damp, then scale by D^-1
    CT a[9];
    const CT dinv[9] = {CT(1) / CT(9),  CT(1) / CT(6),  CT(1) / CT(6),
                        CT(1) / CT(36), CT(1) / CT(36), CT(1) / CT(12),
                        CT(1) / CT(12), CT(1) / CT(4),  CT(1) / CT(4)};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        CT mp = m[i] + k.s[i] * (meq[i] - m[i]);
        if (VAR != kNone) mp += chi * t[i];
        a[i] = mp * dinv[i];
    }

    // g = M^T a
    const CT e1 = a[0] - a[3] - CT(2) * a[4];  // axis populations share this
    const CT e5 = a[0] + CT(2) * a[3] + a[4];  // diagonal populations share this
    const CT x1 = a[1] - CT(2) * a[5], y1 = a[2] - CT(2) * a[6];
    const CT x5 = a[1] + a[5], y5 = a[2] + a[6];
    g[0] = a[0] - CT(4) * a[3] + CT(4) * a[4];
    g[1] = e1 + x1 + a[7];
    g[2] = e1 + y1 - a[7];
    g[3] = e1 - x1 + a[7];
    g[4] = e1 - y1 - a[7];
    g[5] = e5 + x5 + y5 + a[8];
    g[6] = e5 - x5 + y5 - a[8];
    g[7] = e5 - x5 - y5 + a[8];
    g[8] = e5 + x5 - y5 - a[8];
}

// Offsets (in elements, within one plane) of the cells a population is pulled
// from, and whether that cell is inside the lattice.  Population i at (x, y)
// comes from (x - c_ix, y - c_iy).
struct PullSites {
    long long from_xm, from_xp, from_ym, from_yp;  // read x-1, x+1, y-1, y+1
    bool in_xm, in_xp, in_ym, in_yp;

    template <int BC>
    __device__ __forceinline__ void init(int x, int y, const Geometry& g) {
        in_xm = x > 0;
        in_xp = x < g.nx - 1;
        in_ym = y > 0;
        in_yp = y < g.ny - 1;
        from_xm = -1;
        from_xp = 1;
        from_ym = -g.pitch;
        from_yp = g.pitch;
        if (BC == kPeriodic) {
            if (!in_xm) from_xm = g.nx - 1;
            if (!in_xp) from_xp = -(g.nx - 1);
            if (!in_ym) from_ym = (long long)(g.ny - 1) * g.pitch;
            if (!in_yp) from_yp = -(long long)(g.ny - 1) * g.pitch;
        }
    }
    template <int I>
    __device__ __forceinline__ long long offset() const {
        long long o = 0;
        if (cx(I) == 1) o += from_xm;
        if (cx(I) == -1) o += from_xp;
        if (cy(I) == 1) o += from_ym;
        if (cy(I) == -1) o += from_yp;
        return o;
    }
    template <int I>
    __device__ __forceinline__ bool inside() const {
        bool ok = true;
        if (cx(I) == 1) ok = ok && in_xm;
        if (cx(I) == -1) ok = ok && in_xp;
        if (cy(I) == 1) ok = ok && in_ym;
        if (cy(I) == -1) ok = ok && in_yp;
        return ok;
    }
};

// Pull population I of the cell at element offset o (the boundary rule gives
// a zero deviation for Dirichlet far-field walls).
template <typename T, int BC, int I>
__device__ __forceinline__ typename Codec<T>::CT pull(const T* __restrict__ src, long long plane,
                                                      long long o, const PullSites& ps) {
    using CT = typename Codec<T>::CT;
    if (BC == kPeriodic || ps.inside<I>()) {
        return Codec<T>::template dec<I>(__ldg(src + I * plane + o + ps.offset<I>()));
    }
    return CT(0);
}

template <typename T, int BC>
__device__ __forceinline__ void pull_all(const T* __restrict__ src, long long plane, long long o,
                                         const PullSites& ps, typename Codec<T>::CT (&g)[9]) {
    g[0] = pull<T, BC, 0>(src, plane, o, ps);
    g[1] = pull<T, BC, 1>(src, plane, o, ps);
    g[2] = pull<T, BC, 2>(src, plane, o, ps);
    g[3] = pull<T, BC, 3>(src, plane, o, ps);
    g[4] = pull<T, BC, 4>(src, plane, o, ps);
    g[5] = pull<T, BC, 5>(src, plane, o, ps);
    g[6] = pull<T, BC, 6>(src, plane, o, ps);
    g[7] = pull<T, BC, 7>(src, plane, o, ps);
    g[8] = pull<T, BC, 8>(src, plane, o, ps);
}

template <typename T>
__device__ __forceinline__ void store_all(T* __restrict__ dst, long long plane, long long o,
                                          const typename Codec<T>::CT (&g)[9]) {
    dst[0 * plane + o] = Codec<T>::template enc<0>(g[0]);
    dst[1 * plane + o] = Codec<T>::template enc<1>(g[1]);
    dst[2 * plane + o] = Codec<T>::template enc<2>(g[2]);
    dst[3 * plane + o] = Codec<T>::template enc<3>(g[3]);
    dst[4 * plane + o] = Codec<T>::template enc<4>(g[4]);
    dst[5 * plane + o] = Codec<T>::template enc<5>(g[5]);
    dst[6 * plane + o] = Codec<T>::template enc<6>(g[6]);
    dst[7 * plane + o] = Codec<T>::template enc<7>(g[7]);
    dst[8 * plane + o] = Codec<T>::template enc<8>(g[8]);
}

}  // namespace lbm
