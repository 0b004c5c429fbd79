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
//
// Where chi = 0 (the bulk of a lattice) rho* = rho, j* = j and the damping
// term vanishes, so the conserved rows pass through unchanged; the bulk path
// skips that algebra.
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

// FP16 storage keeps q_i = g_i * 2^e_i: a power of two per plane that puts
// g_i / w_i (w = 4/9, 1/9, 1/36) near the middle of the format's range and is
// exact to apply.  BF16 has FP32's exponent range, where such a scale changes
// no rounding (short of FP32 subnormals), so it stores g_i itself.
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
        return __bfloat162float(v);
    }
    template <int I>
    __device__ static __forceinline__ __nv_bfloat16 enc(float v) {
        return __float2bfloat16_rn(v);
    }
};

// ---- Arithmetic on one cell (float, double) or on two packed cells (F2) ----
//
// The collision below is written once over a value type V.  For F2 every
// operation is one packed FP32 instruction (add/sub/mul/fma .rn.f32x2) that
// does the work of two scalar ones; each lane rounds as the scalar
// instruction does (checked on the GPU lane by lane).

// fmadd is one fused multiply-add.  A product written with mul may be fused
// by the compiler into an add that consumes it, in the scalar and in the
// packed form alike (for the packed instructions the code generator does so
// whenever the pattern allows), so the two forms agree to FP32 rounding, not
// bit for bit.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }

__device__ __forceinline__ F2 f2(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.u) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(F2 a) { return __uint_as_float(static_cast<unsigned>(a.u)); }
__device__ __forceinline__ float f2_hi(F2 a) { return __uint_as_float(static_cast<unsigned>(a.u >> 32)); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ F2 fmadd(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(a.u), "l"(b.u), "l"(c.u));
    return r;
}

// A numeric literal in the value type.
template <typename V>
__device__ __forceinline__ V lit(float c) {
    return V(c);
}
template <>
__device__ __forceinline__ F2 lit<F2>(float c) {
    return f2(c, c);
}

// Reciprocal of a value near rho0^2.  FP32: the hardware approximation
// (max 1 ulp); it only scales the |j|^2/rho terms of the equilibrium.
__device__ __forceinline__ float rcp_eq(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_eq(double x) { return __drcp_rn(x); }
__device__ __forceinline__ F2 rcp_eq(F2 x) { return f2(rcp_eq(f2_lo(x)), rcp_eq(f2_hi(x))); }

// Moments m = M g (App. A.1), written as sums and differences.
template <typename V>
__device__ __forceinline__ void moments9(const V (&g)[9], V (&m)[9]) {
    const V a13 = g[1] - g[3], a24 = g[2] - g[4];
    const V b57 = g[5] - g[7], c86 = g[8] - g[6];
    const V p13 = g[1] + g[3], p24 = g[2] + g[4];
    const V p57 = g[5] + g[7], p68 = g[6] + g[8];
    const V s14 = p13 + p24, s58 = p57 + p68;
    const V bpc = b57 + c86, bmc = b57 - c86;
    m[0] = g[0] + s14 + s58;                                 // rho'
    m[1] = a13 + bpc;                                        // j_x'
    m[2] = a24 + bmc;                                        // j_y'
    m[3] = (s58 + s58) - fmadd(lit<V>(4.0f), g[0], s14);     // e: 2 s58 - s14 - 4 g0
    m[4] = fmadd(lit<V>(4.0f), g[0], s58) - (s14 + s14);     // epsilon: 4 g0 - 2 s14 + s58
    m[5] = fmadd(lit<V>(-2.0f), a13, bpc);                   // q_x
    m[6] = fmadd(lit<V>(-2.0f), a24, bmc);                   // q_y
    m[7] = p13 - p24;                                        // p_xx
    m[8] = p57 - p68;                                        // p_xy
}

// m^eq(rho*, j*) - m^eq(rho0, j0) for rows 3, 4, 7, 8 (the nonlinear ones),
// without cancellation:
//   |j*|^2/rho* - |j0|^2/rho0 = (rho0 (|j*|^2 - |j0|^2) - |j0|^2 drho*) / (rho* rho0),
// with |j*|^2 - |j0|^2 = djx (2 jx0 + djx) + djy (2 jy0 + djy).
template <typename V>
__device__ __forceinline__ void quad_eq(V drs, V djx, V djy, const StepConst<V>& k, V& e3, V& e4,
                                        V& e7, V& e8) {
    const V inv = rcp_eq(mul(k.rho0 + drs, k.rho0));
    const V ax = mul(djx, k.jx0_2 + djx);
    const V ay = mul(djy, k.jy0_2 + djy);
    const V q = mul(fmadd(k.njj0, drs, mul(k.rho0, ax + ay)), inv);
    e3 = fmadd(lit<V>(3.0f), q, mul(lit<V>(-2.0f), drs));
    e4 = fmadd(lit<V>(-3.0f), q, drs);
    e7 = mul(fmadd(k.njxy0, drs, mul(k.rho0, ax - ay)), inv);
    // jx* jy* - jx0 jy0 = djx (jy0 + djy) + jx0 djy
    e8 = mul(fmadd(k.npxy0, drs, mul(k.rho0, fmadd(djx, k.jy0 + djy, mul(k.jx0, djy)))), inv);
}

// g = M^T a for a = D^-1 m^+ (the post-collision moments already scaled).
template <typename V>
__device__ __forceinline__ void back9_scaled(const V (&a)[9], V (&g)[9]) {
    const V e1 = fmadd(lit<V>(-2.0f), a[4], a[0] - a[3]);  // shared by the axis populations
    const V e5 = fmadd(lit<V>(2.0f), a[3], a[0] + a[4]);   // shared by the diagonal populations
    const V x1 = fmadd(lit<V>(-2.0f), a[5], a[1]), y1 = fmadd(lit<V>(-2.0f), a[6], a[2]);
    const V x5 = a[1] + a[5], y5 = a[2] + a[6];
    g[0] = fmadd(lit<V>(4.0f), a[4] - a[3], a[0]);
    const V ep = e1 + a[7], em = e1 - a[7];
    g[1] = ep + x1;
    g[3] = ep - x1;
    g[2] = em + y1;
    g[4] = em - y1;
    const V up = e5 + a[8], um = e5 - a[8];
    const V xpy = x5 + y5, xmy = x5 - y5;
    g[5] = up + xpy;
    g[7] = up - xpy;
    g[6] = um - xmy;
    g[8] = um + xmy;
}

// a_k = v / D_k for a conserved row k = 0, 1, 2, correctly rounded (UB): the
// product with 1/D_k rounded once more would scale rho' or j' by 9 fl(1/9) or
// 6 fl(1/6) every step.  16-bit storage rounds each population to 2^-11 or
// 2^-8 on every store, far above that drift, and takes the plain product
// (UB = false), which keeps its kernels at the register count they had.
template <bool UB, typename V>
__device__ __forceinline__ V scale_conserved(V v, const StepConst<V>& k, int row) {
    if (!UB) return mul(v, k.dinv[row]);
    return fmadd(v, k.dinv[row], mul(v, k.dinv_lo[row]));
}

// Whether a storage format takes the correctly rounded conserved scaling.
template <typename T>
struct UnbiasedScale {
    static constexpr bool value = true;
};
template <>
struct UnbiasedScale<__half> {
    static constexpr bool value = false;
};
template <>
struct UnbiasedScale<__nv_bfloat16> {
    static constexpr bool value = false;
};

// Collision where chi = 0: rho* = rho, j* = j, no damping term.  The
// conserved rows are unchanged; the other six relax toward m^eq(rho, j):
// a_k = keep_k m_k + take_k E_k (see StepConst).
template <typename V, bool UB = true>
__device__ __forceinline__ void collide_bulk(V (&g)[9], const StepConst<V>& k) {
    V m[9];
    moments9(g, m);
    V e3, e4, e7, e8;
    quad_eq(m[0], m[1], m[2], k, e3, e4, e7, e8);
    V a[9];
    a[0] = scale_conserved<UB>(m[0], k, 0);
    a[1] = scale_conserved<UB>(m[1], k, 1);
    a[2] = scale_conserved<UB>(m[2], k, 2);
    a[3] = fmadd(k.keep[3], m[3], mul(k.take[3], e3));
    a[4] = fmadd(k.keep[4], m[4], mul(k.take[4], e4));
    a[5] = fmadd(k.keep[5], m[5], mul(k.take[5], m[1]));
    a[6] = fmadd(k.keep[6], m[6], mul(k.take[6], m[2]));
    a[7] = fmadd(k.keep[7], m[7], mul(k.take[7], e7));
    a[8] = fmadd(k.keep[8], m[8], mul(k.take[8], e8));
    back9_scaled(a, g);
}

// The comparison sponge of Sec. 4.1 ("viscosity absorbing"): no damping term,
// and in the layer every non-conserved rate falls linearly toward 1,
// s_k' = s_k + (1 - s_k) r, with r in [0, 1] the layer fraction of the cell.
// Written as the plain relaxation with keep' = (1 - s')/D = keep (1 - r) and
// take' = +-s'/D = take +- keep r, so that r = 0 gives keep and take exactly
// and the result is collide_bulk's bit for bit.
template <typename V, bool UB = true>
__device__ __forceinline__ void collide_viscous(V (&g)[9], V r, const StepConst<V>& k) {
    V m[9];
    moments9(g, m);
    V e3, e4, e7, e8;
    quad_eq(m[0], m[1], m[2], k, e3, e4, e7, e8);
    const V nr = lit<V>(0.0f) - r;
    V kp[9], tp[9];
#pragma unroll
    for (int i = 3; i < 9; ++i) {
        kp[i] = fmadd(k.keep[i], nr, k.keep[i]);
        // rows 5, 6 carry s' with a minus sign (their m^eq is -j)
        tp[i] = fmadd(k.keep[i], (i == 5 || i == 6) ? nr : r, k.take[i]);
    }
    V a[9];
    a[0] = scale_conserved<UB>(m[0], k, 0);
    a[1] = scale_conserved<UB>(m[1], k, 1);
    a[2] = scale_conserved<UB>(m[2], k, 2);
    a[3] = fmadd(kp[3], m[3], mul(tp[3], e3));
    a[4] = fmadd(kp[4], m[4], mul(tp[4], e4));
    a[5] = fmadd(kp[5], m[5], mul(tp[5], m[1]));
    a[6] = fmadd(kp[6], m[6], mul(tp[6], m[2]));
    a[7] = fmadd(kp[7], m[7], mul(tp[7], e7));
    a[8] = fmadd(kp[8], m[8], mul(tp[8], e8));
    back9_scaled(a, g);
}

// Collision with an absorbing strength chi > 0 and its Guo factors rn, rm.
template <typename V, int VAR, bool UB = true>
__device__ __forceinline__ void collide_layer(V (&g)[9], V chi, V rn, V rm,
                                              const StepConst<V>& k) {
    V m[9];
    moments9(g, m);
    // rho*, j*: the Guo definitions solved exactly (sum F = chi (rho_f - rho*),
    // sum c F = chi (j_f - j*)), as deviations from the base state.
    const V drs = mul(fmadd(chi, k.ndrf, m[0]), rn);
    const V djxs = mul(fmadd(chi, k.mdjfx, m[1]), rm);
    const V djys = mul(fmadd(chi, k.mdjfy, m[2]), rm);
    V E[9];  // equilibrium sources (rows 5, 6: j*, the sign is in take)
    E[0] = drs;
    E[1] = djxs;
    E[2] = djys;
    quad_eq(drs, djxs, djys, k, E[3], E[4], E[7], E[8]);
    E[5] = djxs;
    E[6] = djys;

    // T_k of the damping term, times chi
    V ct[9];
    if (VAR == kTypeI) {  // m^eq(q_ref) - m
#pragma unroll
        for (int i = 0; i < 9; ++i) ct[i] = mul(chi, k.dmeq_ref[i] - m[i]);
    } else if (VAR == kTypeII) {  // m^eq(q_ref) - m^eq(rho*, j*)
#pragma unroll
        for (int i = 0; i < 9; ++i)
            ct[i] = mul(chi, (i == 5 || i == 6) ? k.dmeq_ref[i] + E[i] : k.dmeq_ref[i] - E[i]);
    } else {  // type III: linear equilibria (rho, j, -2 rho, rho, -j, 0, 0)
        const V dr = mul(chi, k.drf - drs), dx = mul(chi, k.djfx - djxs), dy = mul(chi, k.djfy - djys);
        const V ndx = mul(chi, djxs - k.djfx), ndy = mul(chi, djys - k.djfy);
        ct[0] = dr;
        ct[1] = dx;
        ct[2] = dy;
        ct[3] = mul(lit<V>(-2.0f), dr);
        ct[4] = dr;
        ct[5] = ndx;
        ct[6] = ndy;
    }
    V a[9];
    // conserved rows: the numerator m + s_c (E - m) + chi T first, then 1/D (with
    // chi = 0: E = m and T = 0, so this is collide_bulk's scaling of m itself)
#pragma unroll
    for (int i = 0; i < 3; ++i)
        a[i] = scale_conserved<UB>(fmadd(k.s[i], E[i] - m[i], m[i]) + ct[i], k, i);
#pragma unroll
    for (int i = 3; i < 9; ++i) {
        if (VAR == kTypeIII && i >= 7)
            a[i] = fmadd(k.keep[i], m[i], mul(k.take[i], E[i]));
        else
            a[i] = fmadd(k.keep[i], m[i], fmadd(k.take[i], E[i], mul(k.dinv[i], ct[i])));
    }
    back9_scaled(a, g);
}

// Per-plane base pointers of one population buffer.
template <typename T>
struct PlanePtrs {
    T* p[9];
};

// Neighbour offsets (elements within a plane) of a cell at (x, y) and whether
// each neighbour is inside the lattice.  Population i at (x, y) is pulled from
// (x - c_ix, y - c_iy).
struct PullSites {
    int from_xm, from_xp, from_ym, from_yp;  // read x-1, x+1, y-1, y+1
    bool in_xm, in_xp, in_ym, in_yp;

    // Interior cells: every neighbour exists, no wrap.
    __device__ __forceinline__ void interior(int pitch) {
        from_xm = -1;
        from_xp = 1;
        from_ym = -pitch;
        from_yp = pitch;
        in_xm = in_xp = in_ym = in_yp = true;
    }
    template <int BC>
    __device__ __forceinline__ void edge(int x, int y, int nx, int ny, int pitch) {
        in_xm = x > 0;
        in_xp = x < nx - 1;
        in_ym = y > 0;
        in_yp = y < ny - 1;
        from_xm = -1;
        from_xp = 1;
        from_ym = -pitch;
        from_yp = pitch;
        if (BC == kPeriodic) {
            if (!in_xm) from_xm = nx - 1;
            if (!in_xp) from_xp = -(nx - 1);
        }
        if (BC == kPeriodic || BC == kChannel) {
            if (!in_ym) from_ym = (ny - 1) * pitch;
            if (!in_yp) from_yp = -(ny - 1) * pitch;
            in_ym = in_yp = true;
        }
        if (BC == kChannel && !in_xp) {  // outflow: the last column's own value
            from_xp = 0;
            in_xp = true;
        }
    }
    template <int I>
    __device__ __forceinline__ int offset() const {
        int o = 0;
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

// Pull population I of the cell at element offset o.  From outside the
// lattice: a Dirichlet far-field wall contributes a zero deviation; the
// channel's source edge contributes src_s * src_e[I] (see LineSource).
// CHECK = false: the cell is interior.
template <typename T, int BC, bool CHECK, int I>
__device__ __forceinline__ typename Codec<T>::CT pull(const PlanePtrs<T>& src, int o,
                                                      const PullSites& ps, double src_s = 0.0,
                                                      const double* src_e = nullptr) {
    using CT = typename Codec<T>::CT;
    if (!CHECK || BC == kPeriodic || ps.inside<I>())
        return Codec<T>::template dec<I>(__ldg(src.p[I] + (o + ps.offset<I>())));
    if (BC == kChannel) return CT(src_s * src_e[I]);  // only cx = +1 at x = 0 gets here
    return CT(0);
}

template <typename T, int BC, bool CHECK>
__device__ __forceinline__ void pull_all(const PlanePtrs<T>& src, int o, const PullSites& ps,
                                         typename Codec<T>::CT (&g)[9], double src_s = 0.0,
                                         const double* src_e = nullptr) {
    g[0] = pull<T, BC, CHECK, 0>(src, o, ps, src_s, src_e);
    g[1] = pull<T, BC, CHECK, 1>(src, o, ps, src_s, src_e);
    g[2] = pull<T, BC, CHECK, 2>(src, o, ps, src_s, src_e);
    g[3] = pull<T, BC, CHECK, 3>(src, o, ps, src_s, src_e);
    g[4] = pull<T, BC, CHECK, 4>(src, o, ps, src_s, src_e);
    g[5] = pull<T, BC, CHECK, 5>(src, o, ps, src_s, src_e);
    g[6] = pull<T, BC, CHECK, 6>(src, o, ps, src_s, src_e);
    g[7] = pull<T, BC, CHECK, 7>(src, o, ps, src_s, src_e);
    g[8] = pull<T, BC, CHECK, 8>(src, o, ps, src_s, src_e);
}

template <typename T>
__device__ __forceinline__ void store_all(const PlanePtrs<T>& dst, int o,
                                          const typename Codec<T>::CT (&g)[9]) {
    dst.p[0][o] = Codec<T>::template enc<0>(g[0]);
    dst.p[1][o] = Codec<T>::template enc<1>(g[1]);
    dst.p[2][o] = Codec<T>::template enc<2>(g[2]);
    dst.p[3][o] = Codec<T>::template enc<3>(g[3]);
    dst.p[4][o] = Codec<T>::template enc<4>(g[4]);
    dst.p[5][o] = Codec<T>::template enc<5>(g[5]);
    dst.p[6][o] = Codec<T>::template enc<6>(g[6]);
    dst.p[7][o] = Codec<T>::template enc<7>(g[7]);
    dst.p[8][o] = Codec<T>::template enc<8>(g[8]);
}

// The same pull and store addressed from one buffer base with 32-bit element
// offsets I * plane + o (valid while 9 planes hold fewer than 2^31 elements);
// keeps two pointers live instead of eighteen.
template <typename T, int BC, bool CHECK, int I>
__device__ __forceinline__ typename Codec<T>::CT pull_b(const T* __restrict__ base, int plane,
                                                        int o, const PullSites& ps) {
    using CT = typename Codec<T>::CT;
    if (!CHECK || BC == kPeriodic || ps.inside<I>())
        return Codec<T>::template dec<I>(
            __ldg(base + static_cast<unsigned>(I * plane + o + ps.offset<I>())));
    return CT(0);
}

template <typename T, int BC, bool CHECK>
__device__ __forceinline__ void pull_all_b(const T* __restrict__ base, int plane, int o,
                                           const PullSites& ps, typename Codec<T>::CT (&g)[9]) {
    g[0] = pull_b<T, BC, CHECK, 0>(base, plane, o, ps);
    g[1] = pull_b<T, BC, CHECK, 1>(base, plane, o, ps);
    g[2] = pull_b<T, BC, CHECK, 2>(base, plane, o, ps);
    g[3] = pull_b<T, BC, CHECK, 3>(base, plane, o, ps);
    g[4] = pull_b<T, BC, CHECK, 4>(base, plane, o, ps);
    g[5] = pull_b<T, BC, CHECK, 5>(base, plane, o, ps);
    g[6] = pull_b<T, BC, CHECK, 6>(base, plane, o, ps);
    g[7] = pull_b<T, BC, CHECK, 7>(base, plane, o, ps);
    g[8] = pull_b<T, BC, CHECK, 8>(base, plane, o, ps);
}

template <typename T>
__device__ __forceinline__ void store_all_b(T* __restrict__ base, int plane, int o,
                                            const typename Codec<T>::CT (&g)[9]) {
    base[static_cast<unsigned>(o)] = Codec<T>::template enc<0>(g[0]);
    base[static_cast<unsigned>(plane + o)] = Codec<T>::template enc<1>(g[1]);
    base[static_cast<unsigned>(2 * plane + o)] = Codec<T>::template enc<2>(g[2]);
    base[static_cast<unsigned>(3 * plane + o)] = Codec<T>::template enc<3>(g[3]);
    base[static_cast<unsigned>(4 * plane + o)] = Codec<T>::template enc<4>(g[4]);
    base[static_cast<unsigned>(5 * plane + o)] = Codec<T>::template enc<5>(g[5]);
    base[static_cast<unsigned>(6 * plane + o)] = Codec<T>::template enc<6>(g[6]);
    base[static_cast<unsigned>(7 * plane + o)] = Codec<T>::template enc<7>(g[7]);
    base[static_cast<unsigned>(8 * plane + o)] = Codec<T>::template enc<8>(g[8]);
}

template <typename T>
__host__ __device__ inline PlanePtrs<T> plane_ptrs(void* base, long long plane) {
    PlanePtrs<T> r;
    for (int i = 0; i < 9; ++i) r.p[i] = static_cast<T*>(base) + i * plane;
    return r;
}

}  // namespace lbm
