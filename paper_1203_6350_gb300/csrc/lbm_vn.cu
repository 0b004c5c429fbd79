// Von Neumann stability maps of the linearised scheme (Secs. 3.2-3.3).
//
// For one "case" (rates S, Guo weights n and m, target velocity u^f, damping
// strength chi, wave direction theta, damping variant) the scheme linearised
// about the uniform state f^eq(rho^f, u^f) advances a plane wave of wave
// vector k by G(k) = diag(exp(-i k.c_i)) J (Eq. sec:matrix).  growth() is the
// largest |lambda| of G(k) over k_j = (pi j / nk)(cos theta, sin theta),
// j = 0..nk; chi_crit() scans chi and bisects on growth > 1 + tol.
//
// J is assembled in moment space, the space the step kernels collide in:
//   M J M^-1 = I - S + S Q - T_m,
// where Q = d m^eq(rho*, j*) / d m (non-zero only in the columns of rho, j_x,
// j_y, through d rho* / d rho = 1/(1 + n chi), d j* / d j = 1/(1 + m chi)),
// and T_m = chi I (type I), chi Q (type II), chi Q_L (type III, the moments of
// the linear equilibrium) or 0.  Then J = M^T D^-1 (M J M^-1) M.
//
// GPU layout: one warp per case.  The warp builds J in shared memory (in FP64,
// then rounded to R), then
// each lane takes wavenumbers lane, lane + 32, ...; for each it forms the
// complex 9 x 9 G(k) in its own shared-memory slot (phases from exp(-i k_x) and
// exp(-i k_y) in R) (element (r, c) of lane l
// at [(9 r + c) * 32 + l], so a warp's accesses fall on consecutive words),
// reduces it to upper Hessenberg form by Householder reflections and finds
// all eigenvalues by the single-shift complex QR iteration with Wilkinson
// shifts and deflation (Golub & Van Loan, Matrix Computations, Secs. 7.4-7.5).
// The arithmetic type R is double or float.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_host.h"

namespace {

constexpr int kVnFields = LBM_VN_FIELDS;
constexpr int kLanes = 32;
constexpr int kN = 9;
constexpr int kMaxIter = 30 * kN;  // QR iterations per matrix before giving up

// D2Q9 velocities and the moment matrix M of App. A.1 (rows: rho, j_x, j_y, e,
// epsilon, q_x, q_y, p_xx, p_xy); D = diag(M M^T).
__constant__ signed char kCx[kN] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ signed char kCy[kN] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ signed char kMat[kN * kN] = {
    1,  1,  1,  1,  1,  1,  1,  1,  1,   //
    0,  1,  0,  -1, 0,  1,  -1, -1, 1,   //
    0,  0,  1,  0,  -1, 1,  1,  -1, -1,  //
    -4, -1, -1, -1, -1, 2,  2,  2,  2,   //
    4,  -2, -2, -2, -2, 1,  1,  1,  1,   //
    0,  -2, 0,  2,  0,  1,  -1, -1, 1,   //
    0,  0,  -2, 0,  2,  1,  1,  -1, -1,  //
    0,  1,  -1, 1,  -1, 0,  0,  0,  0,   //
    0,  0,  0,  0,  0,  1,  -1, 1,  -1};
__constant__ double kDiagD[kN] = {9, 6, 6, 36, 36, 12, 12, 4, 4};

template <typename R>
struct Cx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R a, R b) {
    return Cx<R>{a, b};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) {
    return cx(a.re + b.re, a.im + b.im);
}
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) {
    return cx(a.re - b.re, a.im - b.im);
}
template <typename R>
__device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
    return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__device__ __forceinline__ Cx<R> operator*(R a, Cx<R> b) {
    return cx(a * b.re, a * b.im);
}
template <typename R>
__device__ __forceinline__ Cx<R> conj(Cx<R> a) {
    return cx(a.re, -a.im);
}
// |re| + |im|: the cheap magnitude used by the deflation test.
template <typename R>
__device__ __forceinline__ R abs1(Cx<R> a) {
    return fabs(a.re) + fabs(a.im);
}
template <typename R>
__device__ __forceinline__ R mod(Cx<R> a) {
    return hypot(a.re, a.im);
}
template <typename R>
__device__ __forceinline__ R norm2(Cx<R> a) {
    return a.re * a.re + a.im * a.im;
}
// a / b by Smith's method (R. L. Smith, CACM 5, 1962), which avoids forming |b|^2.
template <typename R>
__device__ __forceinline__ Cx<R> div(Cx<R> a, Cx<R> b) {
    if (fabs(b.re) >= fabs(b.im)) {
        const R r = b.im / b.re, d = b.re + b.im * r;
        return cx((a.re + a.im * r) / d, (a.im - a.re * r) / d);
    }
    const R r = b.re / b.im, d = b.im + b.re * r;
    return cx((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
// Principal square root from sqrt(z) = sqrt((|z| + x)/2) + i y / (2 sqrt(...)),
// taking the branch that avoids cancellation.
template <typename R>
__device__ __forceinline__ Cx<R> csqrt(Cx<R> z) {
    if (z.re == R(0) && z.im == R(0)) return z;
    const R r = hypot(z.re, z.im);
    if (z.re >= R(0)) {
        const R t = sqrt(R(0.5) * (r + z.re));
        return cx(t, z.im / (R(2) * t));
    }
    const R t = sqrt(R(0.5) * (r - z.re));
    return cx(fabs(z.im) / (R(2) * t), copysign(t, z.im));
}

template <typename R>
struct Eps;
template <>
struct Eps<double> {
    static constexpr double v = 2.220446049250313e-16;  // 2^-52
};
template <>
struct Eps<float> {
    static constexpr float v = 1.1920929e-07f;  // 2^-23
};

// Lane-private 9 x 9 complex matrix in shared memory, interleaved across lanes.
template <typename R>
struct Mat {
    Cx<R>* p;  // element (0, 0) of this lane
    __device__ __forceinline__ Cx<R>& operator()(int r, int c) const {
        return p[(r * kN + c) * kLanes];
    }
};

struct Case {
    double s[kN];
    double n, m, ux, uy, theta, chi;
};

__device__ __forceinline__ Case load_case(const double* __restrict__ cases, long long c) {
    const double* q = cases + c * kVnFields;
    Case k;
#pragma unroll
    for (int i = 0; i < kN; ++i) k.s[i] = q[i];
    k.n = q[9];
    k.m = q[10];
    k.ux = q[11];
    k.uy = q[12];
    k.theta = q[13];
    k.chi = q[14];
    return k;
}

// Column c (0 = rho, 1 = j_x, 2 = j_y) of d m^eq / d(rho, j) at u, row r.  The
// moment equilibria of the second-order f^eq are rho, j, e = -2 rho + 3 j^2/rho,
// epsilon = rho - 3 j^2/rho, q = -j, p_xx = (j_x^2 - j_y^2)/rho,
// p_xy = j_x j_y / rho.
__device__ __forceinline__ double dmeq(int r, int c, double ux, double uy) {
    const double uu = ux * ux + uy * uy;
    if (c == 0) {
        const double d[kN] = {1, 0, 0, -2 - 3 * uu, 1 + 3 * uu, 0, 0, -(ux * ux - uy * uy), -ux * uy};
        return d[r];
    }
    if (c == 1) {
        const double d[kN] = {0, 1, 0, 6 * ux, -6 * ux, -1, 0, 2 * ux, uy};
        return d[r];
    }
    const double d[kN] = {0, 0, 1, 6 * uy, -6 * uy, 0, -1, -2 * uy, ux};
    return d[r];
}

// The same for the linear equilibrium w_i (rho + 3 c_i.j): rho, j, e = -2 rho,
// epsilon = rho, q = -j, p = 0.
__device__ __forceinline__ double dmeq_lin(int r, int c) {
    if (c == 0) {
        const double d[kN] = {1, 0, 0, -2, 1, 0, 0, 0, 0};
        return d[r];
    }
    if (c == 1) {
        const double d[kN] = {0, 1, 0, 0, 0, -1, 0, 0, 0};
        return d[r];
    }
    const double d[kN] = {0, 0, 1, 0, 0, 0, -1, 0, 0};
    return d[r];
}

// J of the case at damping strength chi, into jm (scratch) and jp (result),
// 81 doubles each in shared memory.  Called by the whole warp.
__device__ void build_jacobian(const Case& k, int variant, double chi, double* jm, double* jp,
                               int lane) {
    const double a = 1.0 / (1.0 + k.n * chi), b = 1.0 / (1.0 + k.m * chi);
    for (int e = lane; e < kN * kN; e += kLanes) {
        const int r = e / kN, c = e % kN;
        double q = 0.0, ql = 0.0;
        if (c < 3) {
            const double w = c == 0 ? a : b;
            q = w * dmeq(r, c, k.ux, k.uy);
            ql = w * dmeq_lin(r, c);
        }
        double v = (r == c ? 1.0 - k.s[r] : 0.0) + k.s[r] * q;
        if (variant == LBM_SPONGE_I) v -= r == c ? chi : 0.0;
        if (variant == LBM_SPONGE_II) v -= chi * q;
        if (variant == LBM_SPONGE_III) v -= chi * ql;
        jm[e] = v;
    }
    __syncwarp();
    // jp = D^-1 (jm M), row by row
    double x[3];
    int ne = 0;
    for (int e = lane; e < kN * kN; e += kLanes, ++ne) {
        const int r = e / kN, c = e % kN;
        double acc = 0.0;
#pragma unroll
        for (int t = 0; t < kN; ++t) acc += jm[r * kN + t] * kMat[t * kN + c];
        x[ne] = acc / kDiagD[r];
    }
    __syncwarp();
    ne = 0;
    for (int e = lane; e < kN * kN; e += kLanes, ++ne) jp[e] = x[ne];
    __syncwarp();
    // J = M^T jp, back into jm
    ne = 0;
    for (int e = lane; e < kN * kN; e += kLanes, ++ne) {
        const int r = e / kN, c = e % kN;
        double acc = 0.0;
#pragma unroll
        for (int t = 0; t < kN; ++t) acc += kMat[t * kN + r] * jp[t * kN + c];
        x[ne] = acc;
    }
    __syncwarp();
    ne = 0;
    for (int e = lane; e < kN * kN; e += kLanes, ++ne) jp[e] = x[ne];
    __syncwarp();
}

// Reduce A to upper Hessenberg form in place by Householder reflections
// H = I - beta v v^H chosen so that H x = alpha e_1 with |alpha| = |x| and the
// phase of alpha opposite to that of x_1 (no cancellation in v_1).  Entries
// below the subdiagonal are set to exactly zero.
template <typename R>
__device__ void hessenberg(const Mat<R>& A) {
    for (int k = 0; k < kN - 2; ++k) {
        R tail = 0;  // |x|^2 below the subdiagonal
        for (int r = k + 2; r < kN; ++r) tail += norm2(A(r, k));
        if (tail == R(0)) continue;
        const Cx<R> x0 = A(k + 1, k);
        const R ax0 = mod(x0);
        const R nx = sqrt(tail + ax0 * ax0);
        const Cx<R> ph = ax0 > R(0) ? cx(x0.re / ax0, x0.im / ax0) : cx(R(1), R(0));
        const Cx<R> alpha = cx(-ph.re * nx, -ph.im * nx);
        const R big = ax0 + nx;
        A(k + 1, k) = cx(ph.re * big, ph.im * big);  // v_1 = x_1 - alpha; v_r = x_r below
        const R beta = R(2) / (big * big + tail);
        // from the left, on rows k+1.. of columns k+1..
        for (int j = k + 1; j < kN; ++j) {
            Cx<R> s = cx(R(0), R(0));
            for (int r = k + 1; r < kN; ++r) s = s + conj(A(r, k)) * A(r, j);
            s = beta * s;
            for (int r = k + 1; r < kN; ++r) A(r, j) = A(r, j) - A(r, k) * s;
        }
        // from the right, on columns k+1.. of every row
        for (int i = 0; i < kN; ++i) {
            Cx<R> s = cx(R(0), R(0));
            for (int c = k + 1; c < kN; ++c) s = s + A(i, c) * A(c, k);
            s = beta * s;
            for (int c = k + 1; c < kN; ++c) A(i, c) = A(i, c) - s * conj(A(c, k));
        }
        A(k + 1, k) = alpha;
        for (int r = k + 2; r < kN; ++r) A(r, k) = cx(R(0), R(0));
    }
}

// Largest |lambda| of the upper Hessenberg matrix A (destroyed); NaN when the
// QR iteration does not converge within kMaxIter iterations.
//
// Each iteration works on the unreduced block lo..hi: a Wilkinson shift mu (the
// eigenvalue of the trailing 2 x 2 block nearer its last diagonal entry; an
// ad hoc shift every tenth iteration on one eigenvalue), then one implicit
// QR step H - mu I = QR, H <- RQ + mu I by a chase of Givens rotations.  A
// subdiagonal entry below eps (|h_kk| + |h_k-1,k-1|) splits the block; a 1 x 1
// block is an eigenvalue.  Only the active block is updated: the eigenvalues
// do not depend on the rest.
template <typename R>
__device__ R spectral_radius(const Mat<R>& A) {
    const R eps = Eps<R>::v;
    R best = 0;
    int hi = kN - 1, it = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            best = fmax(best, mod(A(0, 0)));
            break;
        }
        int lo = hi;
        while (lo > 0) {
            if (abs1(A(lo, lo - 1)) <= eps * (abs1(A(lo, lo)) + abs1(A(lo - 1, lo - 1)))) {
                A(lo, lo - 1) = cx(R(0), R(0));
                break;
            }
            --lo;
        }
        if (lo == hi) {  // A(hi, hi) is an eigenvalue
            best = fmax(best, mod(A(hi, hi)));
            --hi;
            it = 0;
            continue;
        }
        if (++total > kMaxIter) return R(NAN);
        ++it;
        const Cx<R> a = A(hi - 1, hi - 1), b = A(hi - 1, hi), c = A(hi, hi - 1), d = A(hi, hi);
        Cx<R> mu;
        if (it % 10 == 0) {
            mu = cx(d.re + R(0.75) * abs1(c), d.im);
        } else {
            const Cx<R> p = cx(R(0.5) * (a.re - d.re), R(0.5) * (a.im - d.im));
            const Cx<R> bc = b * c;
            const Cx<R> q = csqrt(p * p + bc);
            const Cx<R> den = abs1(p + q) >= abs1(p - q) ? p + q : p - q;
            mu = (den.re == R(0) && den.im == R(0)) ? d : d - div(bc, den);
        }
        for (int k = lo; k < hi; ++k) {
            Cx<R> x, y;
            if (k == lo) {
                x = A(lo, lo) - mu;
                y = A(lo + 1, lo);
            } else {
                x = A(k, k - 1);
                y = A(k + 1, k - 1);
            }
            // rotation [[cs, sn], [-conj(sn), cs]] taking (x, y) to (r, 0), cs real
            const R ax = mod(x), ay = mod(y);
            R cs;
            Cx<R> sn;
            if (ay == R(0)) {
                cs = R(1);
                sn = cx(R(0), R(0));
            } else if (ax == R(0)) {
                cs = R(0);
                sn = cx(y.re / ay, -y.im / ay);
            } else {
                const R rho = hypot(ax, ay);
                cs = ax / rho;
                sn = cx(x.re / ax, x.im / ax) * cx(y.re / rho, -y.im / rho);
            }
            const Cx<R> nsc = cx(-sn.re, sn.im);  // -conj(sn)
            for (int j = k > lo ? k - 1 : lo; j <= hi; ++j) {
                const Cx<R> t1 = A(k, j), t2 = A(k + 1, j);
                A(k, j) = cs * t1 + sn * t2;
                A(k + 1, j) = nsc * t1 + cs * t2;
            }
            const int last = k + 2 < hi ? k + 2 : hi;
            const Cx<R> snc = conj(sn);
            for (int i = lo; i <= last; ++i) {
                const Cx<R> u1 = A(i, k), u2 = A(i, k + 1);
                A(i, k) = cs * u1 + u2 * snc;
                A(i, k + 1) = cs * u2 - u1 * sn;
            }
            if (k > lo) A(k + 1, k - 1) = cx(R(0), R(0));
        }
    }
    return best;
}

struct Growth {
    double g;  // NaN when an eigenvalue problem did not converge
    double k;  // |k| at the maximum
};

__device__ __forceinline__ void sin_cos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sin_cos(double a, double* s, double* c) { sincos(a, s, c); }

// exp(-i k.c) for c = (cx, cy) in {-1, 0, 1}^2 from ex = exp(-i k_x), ey = exp(-i k_y).
template <typename R>
__device__ __forceinline__ Cx<R> phase(Cx<R> ex, Cx<R> ey, int cxr, int cyr) {
    const Cx<R> one = cx(R(1), R(0));
    const Cx<R> px = cxr > 0 ? ex : (cxr < 0 ? conj(ex) : one);
    const Cx<R> py = cyr > 0 ? ey : (cyr < 0 ? conj(ey) : one);
    return cyr == 0 ? px : (cxr == 0 ? py : px * py);
}

// Largest growth over this lane's wavenumbers, reduced over the warp (every
// lane returns the warp's result).  jr: J (81 values of type R, shared).
template <typename R>
__device__ Growth warp_growth(const R* jr, double theta, int nk, Cx<R>* slot, int lane) {
    const Mat<R> A{slot + lane};
    const double ct = cos(theta), st = sin(theta);
    double g = -1.0, kbest = 0.0;
    bool bad = false;
    for (int j = lane; j <= nk; j += kLanes) {
        const double km = nk > 0 ? 3.141592653589793 * j / nk : 0.0;
        R sx, cxv, sy, cyv;
        sin_cos(static_cast<R>(km * ct), &sx, &cxv);
        sin_cos(static_cast<R>(km * st), &sy, &cyv);
        const Cx<R> ex = cx(cxv, -sx), ey = cx(cyv, -sy);
        for (int r = 0; r < kN; ++r) {
            const Cx<R> ph = phase(ex, ey, kCx[r], kCy[r]);
            for (int c = 0; c < kN; ++c) A(r, c) = jr[r * kN + c] * ph;
        }
        hessenberg(A);
        const double lam = static_cast<double>(spectral_radius(A));
        if (!(lam == lam)) {
            bad = true;
        } else if (lam > g) {
            g = lam;
            kbest = km;
        }
    }
    // warp arg-max, ties to the smaller |k|
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double og = __shfl_xor_sync(0xffffffffu, g, o);
        const double ok = __shfl_xor_sync(0xffffffffu, kbest, o);
        if (og > g || (og == g && ok < kbest)) {
            g = og;
            kbest = ok;
        }
    }
    if (__any_sync(0xffffffffu, bad)) g = NAN;
    return Growth{g, kbest};
}

// J of the case at strength chi, rounded to R, into jr (shared); jm and jp
// are FP64 scratch.  Called by the whole warp.
template <typename R>
__device__ __forceinline__ void jacobian_r(const Case& k, int variant, double chi, double* jm,
                                           double* jp, R* jr, int lane) {
    build_jacobian(k, variant, chi, jm, jp, lane);
    for (int e = lane; e < kN * kN; e += kLanes) jr[e] = static_cast<R>(jp[e]);
    __syncwarp();
}

// Per block: the 32 lane matrices, two FP64 scratch matrices, J in R.
template <typename R>
constexpr size_t vn_smem() {
    return sizeof(Cx<R>) * kN * kN * kLanes + 2 * kN * kN * sizeof(double) +
           kN * kN * sizeof(R);
}

template <typename R>
__global__ void __launch_bounds__(kLanes)
    vn_growth_kernel(const int* __restrict__ variant, const double* __restrict__ cases,
                     int ncases, int nk, double* __restrict__ growth, double* __restrict__ kmax) {
    extern __shared__ __align__(16) unsigned char vn_raw[];
    Cx<R>* slots = reinterpret_cast<Cx<R>*>(vn_raw);
    double* jm = reinterpret_cast<double*>(vn_raw + sizeof(Cx<R>) * kN * kN * kLanes);
    double* jp = jm + kN * kN;
    R* jr = reinterpret_cast<R*>(jp + kN * kN);
    const int lane = threadIdx.x;
    for (long long c = blockIdx.x; c < ncases; c += gridDim.x) {
        const Case k = load_case(cases, c);
        jacobian_r(k, variant[c], k.chi, jm, jp, jr, lane);
        const Growth g = warp_growth<R>(jr, k.theta, nk, slots, lane);
        if (lane == 0) {
            growth[c] = g.g;
            if (kmax) kmax[c] = g.k;
        }
        __syncwarp();
    }
}

template <typename R>
__global__ void __launch_bounds__(kLanes)
    vn_chi_crit_kernel(const int* __restrict__ variant, const double* __restrict__ cases,
                       int ncases, int nk, double chi_lo, double chi_hi, int nscan, int iters,
                       double tol, double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char vn_raw[];
    Cx<R>* slots = reinterpret_cast<Cx<R>*>(vn_raw);
    double* jm = reinterpret_cast<double*>(vn_raw + sizeof(Cx<R>) * kN * kN * kLanes);
    double* jp = jm + kN * kN;
    R* jr = reinterpret_cast<R*>(jp + kN * kN);
    const int lane = threadIdx.x;
    for (long long c = blockIdx.x; c < ncases; c += gridDim.x) {
        const Case k = load_case(cases, c);
        const int var = variant[c];
        // 1: unstable, 0: stable, -1: an eigenvalue problem did not converge
        auto unstable = [&](double chi) -> int {
            jacobian_r(k, var, chi, jm, jp, jr, lane);
            const Growth g = warp_growth<R>(jr, k.theta, nk, slots, lane);
            if (!(g.g == g.g)) return -1;
            return g.g > 1.0 + tol ? 1 : 0;
        };
        double result;
        int u = unstable(chi_lo);
        if (u < 0) {
            result = NAN;
        } else if (u == 1) {
            result = -INFINITY;
        } else {
            double a = chi_lo, b = chi_hi;
            int found = 0;
            for (int g = 1; g < nscan; ++g) {
                const double chi = chi_lo + (chi_hi - chi_lo) * g / (nscan - 1);
                u = unstable(chi);
                if (u != 0) {
                    a = chi_lo + (chi_hi - chi_lo) * (g - 1) / (nscan - 1);
                    b = chi;
                    found = 1;
                    break;
                }
            }
            if (u < 0) {
                result = NAN;
            } else if (!found) {
                result = INFINITY;
            } else {
                for (int i = 0; i < iters && u >= 0; ++i) {
                    const double mid = 0.5 * (a + b);
                    u = unstable(mid);
                    if (u == 1) b = mid;
                    else a = mid;
                }
                result = u < 0 ? NAN : 0.5 * (a + b);
            }
        }
        if (lane == 0) out[c] = result;
        __syncwarp();
    }
}

thread_local std::string g_vn_error;

int fail(int code, const std::string& msg) {
    g_vn_error = msg;
    return code;
}

// Arguments shared by both entry points; returns LBM_OK or LBM_ERR_ARG.
int check_cases(const int* variant, const double* cases, int ncases, int nk, int precision) {
    if (ncases < 0) return fail(LBM_ERR_ARG, "ncases < 0");
    if (nk < 0 || nk > (1 << 24)) return fail(LBM_ERR_ARG, "nk outside [0, 2^24]");
    if (precision != LBM_F64 && precision != LBM_F32)
        return fail(LBM_ERR_ARG, "precision must be LBM_F64 or LBM_F32");
    if (ncases > 0 && (!variant || !cases)) return fail(LBM_ERR_ARG, "NULL case arrays");
    for (long long c = 0; c < ncases; ++c) {
        if (variant[c] < LBM_SPONGE_NONE || variant[c] > LBM_SPONGE_III)
            return fail(LBM_ERR_ARG, "variant must be none, I, II or III");
        const double* q = cases + c * kVnFields;
        for (int f = 0; f < kVnFields; ++f)
            if (!std::isfinite(q[f])) return fail(LBM_ERR_ARG, "non-finite case field");
        if (q[9] < 0 || q[10] < 0 || q[14] < 0)
            return fail(LBM_ERR_ARG, "n, m and chi must be >= 0");
    }
    return LBM_OK;
}

// Device copies of the inputs and room for `nout` doubles of output per case,
// stream-ordered on st.
struct Scratch {
    int* var = nullptr;
    double* cases = nullptr;
    double* out = nullptr;
    cudaStream_t st;
    ~Scratch() {
        if (var) cudaFreeAsync(var, st);
        if (cases) cudaFreeAsync(cases, st);
        if (out) cudaFreeAsync(out, st);
    }
};

int upload(Scratch& s, const int* variant, const double* cases, int ncases, int nout) {
    const size_t nc = static_cast<size_t>(ncases);
    if (cudaMallocAsync(&s.var, nc * sizeof(int), s.st) != cudaSuccess ||
        cudaMallocAsync(&s.cases, nc * kVnFields * sizeof(double), s.st) != cudaSuccess ||
        cudaMallocAsync(&s.out, nc * nout * sizeof(double), s.st) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_OOM, "device allocation failed");
    }
    if (cudaMemcpyAsync(s.var, variant, nc * sizeof(int), cudaMemcpyHostToDevice, s.st) !=
            cudaSuccess ||
        cudaMemcpyAsync(s.cases, cases, nc * kVnFields * sizeof(double), cudaMemcpyHostToDevice,
                        s.st) != cudaSuccess)
        return fail(LBM_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    return LBM_OK;
}

int grid_for(int ncases) {
    return ncases;  // one warp (block) per case
}

template <typename R>
cudaError_t set_smem(const void* fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(vn_smem<R>()));
}

// Copy n doubles of output to the host and wait for the stream.
int finish(Scratch& s, double* dst, size_t n) {
    if (cudaMemcpyAsync(dst, s.out, n * sizeof(double), cudaMemcpyDeviceToHost, s.st) !=
        cudaSuccess)
        return fail(LBM_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    const cudaError_t e = cudaStreamSynchronize(s.st);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}

int nonconverged() { return fail(LBM_ERR_NONFINITE, "an eigenvalue iteration did not converge"); }

}  // namespace

extern "C" {

int lbm_vn_growth(const int* variant, const double* cases, int ncases, int nk, int precision,
                  double* growth, double* k_at_max, void* cuda_stream) {
    const lbm::NvtxRange nvtx("lbm_vn_growth");
    int rc = check_cases(variant, cases, ncases, nk, precision);
    if (rc != LBM_OK) return rc;
    if (ncases > 0 && !growth) return fail(LBM_ERR_ARG, "NULL growth");
    if (ncases == 0) return LBM_OK;
    Scratch s;
    s.st = static_cast<cudaStream_t>(cuda_stream);
    if ((rc = upload(s, variant, cases, ncases, 2)) != LBM_OK) return rc;
    const size_t smem = precision == LBM_F64 ? vn_smem<double>() : vn_smem<float>();
    cudaError_t e;
    if (precision == LBM_F64) {
        e = set_smem<double>(reinterpret_cast<const void*>(vn_growth_kernel<double>));
        if (e == cudaSuccess)
            vn_growth_kernel<double><<<grid_for(ncases), kLanes, smem, s.st>>>(
                s.var, s.cases, ncases, nk, s.out, s.out + ncases);
    } else {
        e = set_smem<float>(reinterpret_cast<const void*>(vn_growth_kernel<float>));
        if (e == cudaSuccess)
            vn_growth_kernel<float><<<grid_for(ncases), kLanes, smem, s.st>>>(
                s.var, s.cases, ncases, nk, s.out, s.out + ncases);
    }
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess)
        return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
    std::vector<double> host(2 * static_cast<size_t>(ncases));
    if ((rc = finish(s, host.data(), host.size())) != LBM_OK) return rc;
    bool nan = false;
    for (int c = 0; c < ncases; ++c) {
        growth[c] = host[c];
        if (k_at_max) k_at_max[c] = host[ncases + c];
        nan = nan || host[c] != host[c];
    }
    return nan ? nonconverged() : LBM_OK;
}

int lbm_vn_chi_crit(const int* variant, const double* cases, int ncases, int nk, int precision,
                    double chi_lo, double chi_hi, int nscan, int iters, double tol,
                    double* chi_crit, void* cuda_stream) {
    const lbm::NvtxRange nvtx("lbm_vn_chi_crit");
    int rc = check_cases(variant, cases, ncases, nk, precision);
    if (rc != LBM_OK) return rc;
    if (!std::isfinite(chi_lo) || !std::isfinite(chi_hi) || chi_lo < 0 || !(chi_hi > chi_lo))
        return fail(LBM_ERR_ARG, "need 0 <= chi_lo < chi_hi, finite");
    if (nscan < 2 || nscan > 4096) return fail(LBM_ERR_ARG, "nscan outside [2, 4096]");
    if (iters < 0 || iters > 200) return fail(LBM_ERR_ARG, "iters outside [0, 200]");
    if (!std::isfinite(tol) || tol < 0) return fail(LBM_ERR_ARG, "tol must be finite and >= 0");
    if (ncases > 0 && !chi_crit) return fail(LBM_ERR_ARG, "NULL chi_crit");
    if (ncases == 0) return LBM_OK;
    Scratch s;
    s.st = static_cast<cudaStream_t>(cuda_stream);
    if ((rc = upload(s, variant, cases, ncases, 1)) != LBM_OK) return rc;
    const size_t smem = precision == LBM_F64 ? vn_smem<double>() : vn_smem<float>();
    cudaError_t e;
    if (precision == LBM_F64) {
        e = set_smem<double>(reinterpret_cast<const void*>(vn_chi_crit_kernel<double>));
        if (e == cudaSuccess)
            vn_chi_crit_kernel<double><<<grid_for(ncases), kLanes, smem, s.st>>>(
                s.var, s.cases, ncases, nk, chi_lo, chi_hi, nscan, iters, tol, s.out);
    } else {
        e = set_smem<float>(reinterpret_cast<const void*>(vn_chi_crit_kernel<float>));
        if (e == cudaSuccess)
            vn_chi_crit_kernel<float><<<grid_for(ncases), kLanes, smem, s.st>>>(
                s.var, s.cases, ncases, nk, chi_lo, chi_hi, nscan, iters, tol, s.out);
    }
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess)
        return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
    if ((rc = finish(s, chi_crit, ncases)) != LBM_OK) return rc;
    for (int c = 0; c < ncases; ++c)
        if (chi_crit[c] != chi_crit[c]) return nonconverged();
    return LBM_OK;
}

const char* lbm_vn_last_error(void) { return g_vn_error.c_str(); }

}  // extern "C"
