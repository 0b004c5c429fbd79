/*
 * FP64 CPU oracle for one time step of the D2Q9 multi-relaxation-time lattice
 * Boltzmann scheme with the absorbing-layer damping terms of Xu & Sagaut,
 * "Analysis of the absorbing layers for the weakly-compressible lattice
 * Boltzmann schemes" (arXiv:1203.6350).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only tests/, the smoke
 * entry point and bench.py's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * The oracle works in POPULATION space, on the full distribution f (not a
 * deviation), with the relaxation matrix Lambda = M^{-1} S M formed explicitly
 * as a 9x9 matrix (Sec. 2.1, Eq. (blbs) and Lambda = M^{-1} S M; App. A.1 for
 * M).  The CUDA path works in moment space on deviations, so the two routes
 * are independent.
 *
 * One time step, per cell x (delta t = 1), following Sec. 2.2:
 *   rho = sum_i f_i,  j = sum_i c_i f_i                              (Eq. q-macro)
 *   chi = max(chi_x[ix], chi_y[iy])                 (corners take the larger strength)
 *   rho* = (rho + n chi rho^f) / (1 + n chi)      (Guo parameterisation, Secs. 2.2.1-2.2.3,
 *   j*   = (j   + m chi rho^f u^f) / (1 + m chi)   solved exactly for rho*, j*, since
 *                                                  sum_i F_i = chi (rho^f - rho*) and
 *                                                  sum_i c_i F_i = chi (j^f - j*), App. B)
 *   fhat_i = f_i + Lambda_ij (f^eq_j(rho*,u*) - f_j) + T_i
 *     type I   (Eq. app:newbgka):       T_i = chi (f^eq_i(rho^f,u^f) - f_i)
 *     type II  (Eq. app:newbgka2):      T_i = chi (f^eq_i(rho^f,u^f) - f^eq_i(rho*,u*))
 *     type III (Eq. app:bgk_no2ordor2): T_i = chi (f^Leq_i(rho^f,j^f) - f^Leq_i(rho*,j*))
 *     none:                             T_i = 0, and chi = 0 (no absorbing term at all)
 *   The comparison strategy of Sec. 4.1 (viscosity sponge, variant 4) has no
 *   damping term and relaxation rates that fall to 1 across the layer; see
 *   oracle_collide_cell_viscous.
 *   f_i(x + c_i, t + 1) = fhat_i(x, t)                               (Eq. blbs)
 *
 * Readings of points the paper leaves open:
 *   - f^eq is the standard second-order D2Q9 equilibrium
 *       f^eq_i = w_i rho (1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u)
 *     and its linear part is f^Leq_i(rho, j) = w_i (rho + 3 c_i.j).
 *   - rho*, j* are the implicit (exact) solution of the Guo definitions.
 *   - S carries a rate s_c on the conserved rows 0..2 (s[0..2]); with all
 *     nine rates equal the scheme is the paper's BGK scheme.
 *   - Boundary "Dirichlet far field": a population that would stream in from
 *     outside the lattice takes the value f^eq_i(rho0, u0).  This holds at
 *     every time level including t = 0 (oracle_init applies it).
 *   - Periodic: the lattice wraps in both directions.
 *   - Channel (the time-dependent line source of Sec. 4.2): periodic in y; at
 *     the left edge a population streaming in from x = -1 takes the value of
 *     the equilibrium f^eq_i(rho_s(t), u0) with rho_s(t) = rho0 + A sin(w t +
 *     phi), t the time of the post-collision state it leaves; at the right
 *     edge (outflow) a population streaming in from x = nx takes the
 *     post-collision value of the same population at x = nx - 1 (zero
 *     gradient).  At t = 0 (oracle_init) the left edge takes rho_s(-1) and the
 *     right edge the equilibrium of the initial state at x = nx - 2.
 *
 * Layout: f[(i * ny + iy) * nx + ix], i = 0..8 in the velocity order fixed by
 * rows 1-2 of M (App. A.1): c = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
 * (-1,-1),(1,-1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny;
    int bc;        /* 0: Dirichlet far-field equilibrium, 1: periodic, 2: channel */
    int variant;   /* 0: none, 1: type I, 2: type II, 3: type III, 4: viscosity sponge */
    double rho0, ux0, uy0;    /* far-field state of the boundary */
    double rho_f, ux_f, uy_f; /* reference state q_ref of the absorbing term */
    double s[9];   /* diagonal of S in the row order of M */
    double n, m;   /* weights of the Guo parameterisation */
    double src_amp, src_omega, src_phase;  /* channel: rho_s(t) = rho0 + A sin(w t + phi) */
    double t0;     /* time of the state oracle_run starts from */
} oracle_params;

static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WGT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Transformation matrix of App. A.1, row by row. */
static const double MMAT[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
};

/* Copies of the tables for the tests (so they can check the oracle's own data). */
void oracle_tables(int* cx, int* cy, double* w, double* mmat) {
    for (int i = 0; i < 9; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = WGT[i];
        for (int j = 0; j < 9; ++j) mmat[i * 9 + j] = MMAT[i][j];
    }
}

/* f^eq_i(rho, u): second-order equilibrium, c_s^2 = 1/3. */
void oracle_feq(double rho, double ux, double uy, double* out) {
    const double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        const double cu = CX[i] * ux + CY[i] * uy;
        out[i] = WGT[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* f^Leq_i(rho, j): the part of f^eq that is linear in (rho, j). */
void oracle_feq_linear(double rho, double jx, double jy, double* out) {
    for (int i = 0; i < 9; ++i) out[i] = WGT[i] * (rho + 3.0 * (CX[i] * jx + CY[i] * jy));
}

/* Inverse of a 9x9 matrix by Gauss-Jordan elimination with partial pivoting.
 * Returns 0 on success, -1 if singular. */
static int invert9(const double a_in[9][9], double inv[9][9]) {
    double a[9][18];
    for (int i = 0; i < 9; ++i) {
        for (int j = 0; j < 9; ++j) {
            a[i][j] = a_in[i][j];
            a[i][9 + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (fabs(a[piv][col]) < 1e-300) return -1;
        if (piv != col)
            for (int j = 0; j < 18; ++j) {
                double t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        const double d = a[col][col];
        for (int j = 0; j < 18; ++j) a[col][j] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == col) continue;
            const double fct = a[r][col];
            if (fct == 0.0) continue;
            for (int j = 0; j < 18; ++j) a[r][j] -= fct * a[col][j];
        }
    }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) inv[i][j] = a[i][9 + j];
    return 0;
}

/* Lambda = M^{-1} diag(s) M (Sec. 2.1), written to out[9*9] row-major. */
int oracle_lambda(const double* s, double* out) {
    double minv[9][9];
    if (invert9(MMAT, minv) != 0) return -1;
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 9; ++k) acc += minv[i][k] * s[k] * MMAT[k][j];
            out[i * 9 + j] = acc;
        }
    return 0;
}

/* Post-collision populations of one cell (the right-hand side of Eq. blbs-abc-1
 * with Gamma = chi I), for the chosen damping variant. */
void oracle_collide_cell(const oracle_params* p, const double* lam, double chi, const double* f,
                         double* fhat) {
    /* Without a damping term Gamma = 0, so F = 0 and rho* = rho, j* = j (Eq. blbs). */
    if (p->variant == 0) chi = 0.0;
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    const double jfx = p->rho_f * p->ux_f, jfy = p->rho_f * p->uy_f;
    const double rs = (rho + p->n * chi * p->rho_f) / (1.0 + p->n * chi);
    const double jxs = (jx + p->m * chi * jfx) / (1.0 + p->m * chi);
    const double jys = (jy + p->m * chi * jfy) / (1.0 + p->m * chi);
    double fs[9], d[9], t[9];
    oracle_feq(rs, jxs / rs, jys / rs, fs);
    for (int i = 0; i < 9; ++i) d[i] = fs[i] - f[i];

    for (int i = 0; i < 9; ++i) t[i] = 0.0;
    if (p->variant == 1) {
        double fr[9];
        oracle_feq(p->rho_f, p->ux_f, p->uy_f, fr);
        for (int i = 0; i < 9; ++i) t[i] = chi * (fr[i] - f[i]);
    } else if (p->variant == 2) {
        double fr[9];
        oracle_feq(p->rho_f, p->ux_f, p->uy_f, fr);
        for (int i = 0; i < 9; ++i) t[i] = chi * (fr[i] - fs[i]);
    } else if (p->variant == 3) {
        double lr[9], ls[9];
        oracle_feq_linear(p->rho_f, jfx, jfy, lr);
        oracle_feq_linear(rs, jxs, jys, ls);
        for (int i = 0; i < 9; ++i) t[i] = chi * (lr[i] - ls[i]);
    }
    for (int i = 0; i < 9; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 9; ++j) acc += lam[i * 9 + j] * d[j];
        fhat[i] = f[i] + acc + t[i];
    }
}

/* The comparison strategy of Sec. 4.1 ("viscosity absorbing"): no damping
 * term; in the layer the relaxation frequency falls linearly from its
 * physical value to 1.  With the layer fraction r in [0, 1] (0 at the inner
 * edge, 1 at the wall) every non-conserved rate becomes
 * s_k' = s_k + (1 - s_k) r, so Lambda' = (1 - r) Lambda + r Lambda1 with
 * Lambda1 = M^{-1} diag(s_0, s_1, s_2, 1, ..., 1) M.  rho, j are unchanged by
 * the collision (no forcing, rho* = rho). */
void oracle_collide_cell_viscous(const oracle_params* p, const double* lam, const double* lam1,
                                 double r, const double* f, double* fhat) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double fs[9];
    oracle_feq(rho, jx / rho, jy / rho, fs);
    (void)p;
    for (int i = 0; i < 9; ++i) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < 9; ++j) {
            a += lam[i * 9 + j] * (fs[j] - f[j]);
            b += lam1[i * 9 + j] * (fs[j] - f[j]);
        }
        fhat[i] = f[i] + (1.0 - r) * a + r * b;
    }
}

static inline size_t idx(const oracle_params* p, int i, int iy, int ix) {
    return ((size_t)i * p->ny + iy) * p->nx + ix;
}

/* Density of the line source at time t (channel boundary). */
static double source_rho(const oracle_params* p, double t) {
    return p->rho0 + p->src_amp * sin(p->src_omega * t + p->src_phase);
}

/* Initial state: f = f^eq(rho(x), u(x)) at every cell, then the boundary rule
 * for populations entering from outside (Dirichlet and channel).  rho, ux, uy
 * are [ny][nx] row-major. */
int oracle_init(const oracle_params* p, const double* rho, const double* ux, const double* uy,
                double* f) {
    const int nx = p->nx, ny = p->ny;
    if (nx <= 0 || ny <= 0) return -1;
    if (p->bc == 2 && nx < 2) return -1;
    double fb[9], fs[9];
    oracle_feq(p->rho0, p->ux0, p->uy0, fb);
    oracle_feq(source_rho(p, p->t0 - 1.0), p->ux0, p->uy0, fs);
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) {
            double fe[9], fo[9];
            const size_t c = (size_t)iy * nx + ix;
            oracle_feq(rho[c], ux[c], uy[c], fe);
            if (p->bc == 2 && ix == nx - 1) {  /* zero gradient: the column inside */
                const size_t c2 = (size_t)iy * nx + ix - 1;
                oracle_feq(rho[c2], ux[c2], uy[c2], fo);
            }
            for (int i = 0; i < 9; ++i) {
                const int sx = ix - CX[i], sy = iy - CY[i];
                const int outside = sx < 0 || sx >= nx || sy < 0 || sy >= ny;
                double v = fe[i];
                if (p->bc == 0 && outside) v = fb[i];
                if (p->bc == 2 && sx < 0) v = fs[i];
                if (p->bc == 2 && sx >= nx) v = fo[i];
                f[idx(p, i, iy, ix)] = v;
            }
        }
    return 0;
}

/* Advance f by nsteps time steps.  chi_x has nx entries, chi_y has ny.
 * nthreads <= 0 means the OpenMP default. */
int oracle_run(const oracle_params* p, const double* chi_x, const double* chi_y, double* f,
               int nsteps, int nthreads) {
    const int nx = p->nx, ny = p->ny;
    if (nx <= 0 || ny <= 0 || nsteps < 0) return -1;
    double lam[81], lam1[81], s1[9];
    if (oracle_lambda(p->s, lam) != 0) return -2;
    for (int k = 0; k < 9; ++k) s1[k] = k < 3 ? p->s[k] : 1.0;
    if (oracle_lambda(s1, lam1) != 0) return -2;
    if (p->bc == 2 && nx < 2) return -1;
    double fb[9];
    oracle_feq(p->rho0, p->ux0, p->uy0, fb);
    const size_t ncell = (size_t)nx * ny;
    double* post = (double*)malloc(sizeof(double) * 9 * ncell);
    if (!post) return -3;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    (void)nthreads;
#endif
    for (int step = 0; step < nsteps; ++step) {
        /* collision at every cell */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
        for (int iy = 0; iy < ny; ++iy) {
            for (int ix = 0; ix < nx; ++ix) {
                double fc[9], fh[9];
                for (int i = 0; i < 9; ++i) fc[i] = f[idx(p, i, iy, ix)];
                const double chi = chi_x[ix] > chi_y[iy] ? chi_x[ix] : chi_y[iy];
                if (p->variant == 4)  /* the arrays carry the layer fraction r */
                    oracle_collide_cell_viscous(p, lam, lam1, chi, fc, fh);
                else
                    oracle_collide_cell(p, lam, chi, fc, fh);
                for (int i = 0; i < 9; ++i) post[idx(p, i, iy, ix)] = fh[i];
            }
        }
        /* streaming: f_i(x) = fhat_i(x - c_i) */
        double fs[9];  /* channel: the source column's post-collision state at this time */
        oracle_feq(source_rho(p, p->t0 + step), p->ux0, p->uy0, fs);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
        for (int iy = 0; iy < ny; ++iy) {
            for (int ix = 0; ix < nx; ++ix) {
                for (int i = 0; i < 9; ++i) {
                    int sx = ix - CX[i], sy = iy - CY[i];
                    double v;
                    if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) {
                        v = post[idx(p, i, sy, sx)];
                    } else if (p->bc == 1) {
                        sx = (sx + nx) % nx;
                        sy = (sy + ny) % ny;
                        v = post[idx(p, i, sy, sx)];
                    } else if (p->bc == 2) {
                        sy = (sy + ny) % ny;
                        if (sx < 0)
                            v = fs[i];
                        else if (sx >= nx)
                            v = post[idx(p, i, sy, nx - 1)];
                        else
                            v = post[idx(p, i, sy, sx)];
                    } else {
                        v = fb[i];
                    }
                    f[idx(p, i, iy, ix)] = v;
                }
            }
        }
    }
    free(post);
    return 0;
}

/* Macroscopic fields of the state f: rho - rho0, u_x, u_y as [ny][nx]. */
void oracle_moments(const oracle_params* p, const double* f, double* rho_dev, double* ux,
                    double* uy) {
    const int nx = p->nx, ny = p->ny;
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) {
            double rho = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                const double v = f[idx(p, i, iy, ix)];
                rho += v;
                jx += CX[i] * v;
                jy += CY[i] * v;
            }
            const size_t c = (size_t)iy * nx + ix;
            rho_dev[c] = rho - p->rho0;
            ux[c] = jx / rho;
            uy[c] = jy / rho;
        }
}
