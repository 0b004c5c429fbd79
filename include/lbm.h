/*
 * lbm.h -- C ABI of the GB300 (sm_103a) time step of the weakly-compressible
 * D2Q9 multi-relaxation-time lattice Boltzmann scheme with the absorbing-layer
 * damping terms of Xu & Sagaut, "Analysis of the absorbing layers for the
 * weakly-compressible lattice Boltzmann schemes" (arXiv:1203.6350).
 *
 * The scheme (Sec. 2, Eq. blbs-abc-1 with Gamma = chi I, Eq. eq:gamma):
 *
 *   f_i(x + c_i, t + 1) = f_i + Lambda_ij (f^eq_j(rho*, u*) - f_j)
 *                         + chi(x) (f^ref_i - f*_i),       Lambda = M^-1 S M,
 *
 * with three choices of (f^ref, f*) (Secs. 2.2.1-2.2.3): type I f^eq(q_ref)
 * and f; type II f^eq(q_ref) and f^eq(rho*, u*); type III the linear
 * equilibria of both.  rho*, j* = rho* u* follow the Guo parameterisation
 * with weights n, m, solved exactly:
 *   rho* = (rho + n chi rho_ref) / (1 + n chi),  j* = (j + m chi j_ref) / (1 + m chi).
 * The velocity set and M are those of App. A.1:
 *   c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - delta t = 1, lattice units, c_s^2 = 1/3.
 *  - Fields passed in or out are FP64, [ny][nx] row-major (x fastest).
 *  - The lattice is double-buffered in device memory as 9 planes per buffer
 *    of populations stored as DEVIATIONS g_i = f_i - f^eq_i(rho0, u0) from the
 *    far-field state given to lbm_create (FP64, FP32, FP16 with a fixed
 *    power-of-two scale per plane, or BF16).
 *  - "Time" counts steps; lbm_init_equilibrium sets time 0.
 *  - Boundary: LBM_BC_DIRICHLET_EQ makes every population that would stream
 *    in from outside equal to f^eq(rho0, u0), at every time level including
 *    t = 0; LBM_BC_PERIODIC wraps both axes.
 *  - Calls that launch work are asynchronous on the handle's stream unless
 *    they say they synchronise.  Calls on one handle must not overlap from
 *    several host threads.
 *
 * Return codes: LBM_OK (0); a positive value is a warning (the call did its
 * work); a negative value is an error (the call did nothing unless it says
 * otherwise).  lbm_last_error() gives a message for the last non-zero code.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx* lbm_handle;

/* Storage of the populations.  F16DEV / BF16DEV keep 16-bit deviations; the
 * arithmetic is FP32 for every storage but F64. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16DEV = 2, LBM_BF16DEV = 3 } lbm_storage;

/* Damping term (Sec. 2.2): none, type I (Eq. app:newbgka), type II
 * (Eq. app:newbgka2), type III (Eq. app:bgk_no2ordor2).  LBM_SPONGE_VISCOUS
 * is the comparison strategy of Sec. 4.1 ("viscosity absorbing"): no damping
 * term; in the layer every non-conserved relaxation rate falls linearly from
 * its value to 1, s_k' = s_k + (1 - s_k) r, where r in [0, 1] is the layer
 * fraction taken from the same per-axis arrays as chi (r = max of the two). */
typedef enum {
    LBM_SPONGE_NONE = 0,
    LBM_SPONGE_I = 1,
    LBM_SPONGE_II = 2,
    LBM_SPONGE_III = 3,
    LBM_SPONGE_VISCOUS = 4
} lbm_variant;

/* Boundary.  LBM_BC_CHANNEL is the acoustic line-source case of Sec. 4.2:
 * periodic in y; a population entering at the left edge (x = 0) is that of
 * the equilibrium f^eq(rho_s(t), u0) of the source column, rho_s(t) = rho0 +
 * A sin(omega t + phase) (lbm_set_source; A = 0 until set), t the time of the
 * post-collision state it leaves (so the state of time 0 takes rho_s(-1));
 * a population entering at the right edge (outflow, x = nx - 1) takes the
 * post-collision value of the same population of the last column (zero
 * gradient), and at time 0 the initial equilibrium of the column x = nx - 2.
 * Single lattices only (lbm_batch_add rejects it); one step per launch. */
typedef enum { LBM_BC_DIRICHLET_EQ = 0, LBM_BC_PERIODIC = 1, LBM_BC_CHANNEL = 2 } lbm_bc;

/* Relaxation rates: s[k] is the diagonal of S in the row order of M
 * (App. A.1): s[0..2] act on the conserved rows rho, j_x, j_y (rate s_c,
 * which multiplies rho* - rho and j* - j), s[3] = s_e, s[4] = s_eps,
 * s[5..6] = s_q, s[7..8] = s_nu.  All nine equal gives the BGK scheme the
 * paper analyses.  n, m are the weights of the Guo parameterisation. */
typedef struct {
    double s[9];
    double n;
    double m;
} lbm_rates;

/* Optional device allocator.  alloc returns a device pointer (>= 256-byte
 * aligned) or NULL; free releases it.  ctx is passed back unchanged.  The
 * library calls them inside lbm_create, lbm_destroy, and the first
 * lbm_init_equilibrium / lbm_moments that uses host buffers (a staging area
 * of 24 bytes per cell, kept until lbm_destroy). */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* ctx);
    void* ctx;
} lbm_allocator;

#define LBM_OK 0
#define LBM_WARN_UNSTABLE_PARAMS 1 /* chi > 4/s (type II/III), s + chi > 2 (type I), s_k outside (0, 2) */
#define LBM_ERR_ARG (-1)           /* bad argument: nothing was done */
#define LBM_ERR_OOM (-2)           /* device allocation failed */
#define LBM_ERR_CUDA (-3)          /* a CUDA call failed; see lbm_last_error */
#define LBM_ERR_NONFINITE (-4)     /* the state holds NaN or Inf (diagnostics found it) */
#define LBM_ERR_STATE (-5)         /* call out of order (e.g. step before init) */

/* Create a lattice of nx * ny cells (1 <= nx, ny; nx * ny <= 2^31 - 1) with
 * far-field state (rho0 > 0, u0) -- the deviation base and the Dirichlet
 * boundary state -- relaxation rates *rates (Sec. 2.1), boundary bc, on the
 * CUDA stream cuda_stream (a cudaStream_t, borrowed; NULL = legacy default
 * stream).  alloc = NULL uses cudaMalloc / cudaFree.  The damping term is
 * off until lbm_set_sponge.  On success *out owns two population buffers of
 * 9 * ny * pitch elements each (pitch = nx rounded up to 128 bytes).
 * Returns LBM_WARN_UNSTABLE_PARAMS if some s_k is outside (0, 2) (the paper's
 * constraint, Sec. 2.1), LBM_ERR_ARG, LBM_ERR_OOM or LBM_ERR_CUDA. */
int lbm_create(int nx, int ny, lbm_storage storage, double rho0, double ux0, double uy0,
               const lbm_rates* rates, lbm_bc bc, void* cuda_stream, const lbm_allocator* alloc,
               lbm_handle* out);

/* Set the damping term: variant, per-axis strengths chi_x[nx], chi_y[ny]
 * (host arrays, >= 0, copied; the strength at cell (ix, iy) is
 * max(chi_x[ix], chi_y[iy])), and the reference state q_ref = (rho_ref,
 * u_ref) of Eq. (eq:reff).  Takes effect from the next lbm_step.
 * Returns LBM_WARN_UNSTABLE_PARAMS when max chi exceeds the paper's critical
 * value (4/s_nu for types II and III, Eq. criticalchi; 2 - s_nu for type I,
 * Eq. effectrelax), LBM_ERR_ARG for NULL / negative / non-finite input. */
int lbm_set_sponge(lbm_handle h, lbm_variant variant, const double* chi_x, const double* chi_y,
                   double rho_ref, double ux_ref, double uy_ref);

/* Time 0: f = f^eq(rho(x), u(x)) at every cell (Sec. 4.1 initialises the
 * pulse at equilibrium), then the boundary rule.  rho, ux, uy are FP64
 * [ny][nx]; on_device != 0 means they are device pointers (read on the
 * handle's stream), else host pointers (copied; the call synchronises the
 * stream).  Resets the step counter. */
int lbm_init_equilibrium(lbm_handle h, const double* rho, const double* ux, const double* uy,
                         int on_device);

/* Time 0 of the 2-D acoustic pulse of Sec. 4.1 (Eqs. pulseprofile, 3:para0),
 * built on the device with no input field: rho = rho0 + eps exp(-alpha r^2),
 * alpha = ln 2 / half_width^2, r the distance of the cell (ix, iy) from
 * (x0, y0), u = u0, f = f^eq(rho, u), then the boundary rule.  Asynchronous;
 * resets the step counter.  LBM_ERR_ARG for non-finite input or
 * half_width <= 0. */
int lbm_init_pulse(lbm_handle h, double eps, double half_width, double x0, double y0);

/* Advance nsteps >= 0 time steps: one fused kernel per step (pull-stream,
 * moments, rho* and j*, MRT relaxation, damping term, back-transform,
 * store), asynchronous on the handle's stream. */
int lbm_step(lbm_handle h, int nsteps);

/* Fields at the current time: rho_dev = rho - rho0, ux, uy (FP64 [ny][nx];
 * any pointer may be NULL to skip it).  on_device != 0: device pointers,
 * asynchronous; else host pointers and the call synchronises. */
int lbm_moments(lbm_handle h, double* rho_dev, double* ux, double* uy, int on_device);

/* FP64 reductions over the cells x0 <= ix < x1, y0 <= iy < y1 at the current
 * time (host out[6], synchronises):
 *   out[0] sum rho'           out[1] sum (j_x - rho0 u0x)   out[2] sum (j_y - rho0 u0y)
 *   out[3] acoustic energy sum [c_s^2 rho'^2 / (2 rho0) + rho0 |u - u0|^2 / 2]
 *   out[4] sum rho'^2 (numerator of E_L2, Sec. 4.1, with rho_ref = rho0)
 *   out[5] number of cells with a non-finite rho' or u
 * Returns LBM_ERR_NONFINITE (with out filled) when out[5] > 0. */
int lbm_diagnostics(lbm_handle h, int x0, int y0, int x1, int y1, double out[6]);

/* Checkpoint: the raw population buffer of the current time (bytes =
 * lbm_state_bytes) and the step counter.  on_device selects device or host
 * memory for dst/src; host transfers synchronise.  The buffer holds 9 planes
 * of ny rows of pitch elements (pitch = nx rounded up to 128 bytes).
 *
 * Padding canaries (a debugging aid): with the environment variable
 * LBM_CANARY=1 at lbm_create (lbm_batch_create, lbm3_create), the padding of
 * every row -- elements nx .. pitch - 1 -- of both population buffers is set
 * to all-one bytes, a NaN in every storage format.  No kernel reads or writes
 * padding, so the padding of the state returned here stays all-one bytes and
 * the cells' values equal those of a run without canaries. */
size_t lbm_state_bytes(lbm_handle h);
int lbm_get_state(lbm_handle h, void* dst, size_t bytes, int on_device, int64_t* time);
int lbm_set_state(lbm_handle h, const void* src, size_t bytes, int on_device, int64_t time);

/* Steps taken since lbm_init_equilibrium (or set by lbm_set_state). */
int64_t lbm_time(lbm_handle h);

/* How lbm_step issues its kernels: 0 one launch per step; 1 one launch per
 * step, each a programmatic dependent of the previous (its launch overlaps
 * the previous step's tail); 2 (default) replays of a captured graph of 64
 * steps of such launches (64 one-step or 32 two-step launches), with single
 * launches for the remainder.  All three compute identical results.  The environment variable LBM_LAUNCH=plain|pdl|graph
 * sets the initial mode of new handles. */
int lbm_set_launch_mode(lbm_handle h, int mode);

/* Cells each thread of the step kernel advances: 1, or 2 -- the neighbouring
 * cells (x, x + 1) stepped together with packed two-lane FP32 arithmetic and
 * paired loads and stores.  2 is available for LBM_F32, LBM_F16DEV and
 * LBM_BF16DEV storage while the nine population planes hold fewer than 2^32
 * elements, and is then the default; otherwise (and for LBM_F64) 1.  Both
 * evaluate the same collision in the same order; they agree to FP32
 * rounding (the code generator may fuse a product into the add that
 * consumes it in one form and not in the other).  LBM_ERR_ARG for any other
 * value or an unsupported 2.  Waits for the handle's stream.  The environment
 * variable LBM_CPT=1 makes 1 the initial choice of new handles. */
int lbm_set_cells_per_thread(lbm_handle h, int cells);
/* The current choice (LBM_ERR_ARG for a NULL handle). */
int lbm_cells_per_thread(lbm_handle h);

/* Time steps per kernel launch: 1, or 2 -- temporal blocking.  With 2 each
 * launch reads the state of time t from HBM once, computes time t + 1 on its
 * tile and a one-cell ring around it in shared memory (stored there in the
 * handle's storage format, as a one-step launch would store it in HBM), and
 * writes time t + 2: half the HBM traffic per step for 1.2 times the
 * collisions.  Needs two cells per thread (lbm_set_cells_per_thread(h, 1)
 * switches it back to 1).  lbm_step(h, n) then issues n / 2 two-step
 * launches and one one-step launch for an odd n.  Results agree with one step
 * per launch to FP32 rounding.  LBM_ERR_ARG for any other value or an
 * unsupported 2.  Waits for the handle's stream.  New handles start with 2
 * where it is available and the two population buffers together exceed the
 * device's L2 cache (the step is then HBM-bound), else 1; the environment
 * variable LBM_SPL=1|2 overrides that choice. */
int lbm_set_steps_per_launch(lbm_handle h, int steps);
/* The current choice (LBM_ERR_ARG for a NULL handle). */
int lbm_steps_per_launch(lbm_handle h);

/* Arithmetic of the collision (Sec. 2, Eq. blbs-abc-1; the same step, only the
 * rounding differs).  LBM_ARITH_NATIVE (the default): FP64 for LBM_F64
 * storage, FP32 otherwise.  LBM_ARITH_COMPENSATED (LBM_F32 storage only):
 * the populations stay FP32 in memory, but the collision runs in float-float
 * arithmetic -- each value carried as an unevaluated sum of two FP32 numbers,
 * each operation built from error-free FP32 transformations (Knuth's TwoSum,
 * Dekker's Fast2Sum, a fused-multiply-add product) -- about 44 correct bits,
 * so the only per-step rounding left is the FP32 store.  Where a field decays
 * by orders of magnitude (an absorbed pulse) the FP32 collision's own
 * roundings, ~10 per population per step, dominate its error against an
 * FP64 reference; the compensated step removes them at several times the
 * FP32 kernel's instruction count (still on FP32 pipes, far above GB300's
 * FP64 rate).  It steps one cell, one time step per launch: while it is
 * selected, lbm_set_cells_per_thread(h, 2), lbm_set_steps_per_launch(h, 2)
 * and lbm_set_tma_staging(h, 1) return LBM_ERR_ARG; selecting it sets one
 * cell and one step per launch.  LBM_ERR_ARG for other values or storage.
 * Waits for the handle's stream.  lbm_get_arithmetic returns the current choice
 * (LBM_ERR_ARG for a NULL handle). */
typedef enum { LBM_ARITH_NATIVE = 0, LBM_ARITH_COMPENSATED = 1 } lbm_arithmetic;
int lbm_set_arithmetic(lbm_handle h, lbm_arithmetic a);
int lbm_get_arithmetic(lbm_handle h);

/* Staging of the two-step launches' input by the Tensor Memory Accelerator.
 * With it (1), each 64 x 16 tile's input -- the nine planes of the 72 x 20
 * cells around it -- arrives in shared memory as one bulk tensor copy whose
 * out-of-lattice elements read as zero (the Dirichlet far-field deviation);
 * the copy of a CTA's next tile overlaps the current tile's second step.
 * The results are bit-identical to those without it (0).  Available for
 * LBM_F32, LBM_F16DEV and LBM_BF16DEV storage with LBM_BC_DIRICHLET_EQ (a
 * 72 x 20 box of FP32, or 80 x 20 of 16-bit elements, starting 16 bytes left
 * of the tile); the default for LBM_F32 where both population buffers
 * together exceed four times the L2 size (the environment variable LBM_TMA=0
 * or 1 at lbm_create overrides that choice; 16-bit storage measured level
 * with plain loads and is not staged by default); LBM_ERR_ARG for other
 * handles or values.  A staged copy that has not
 * completed after a bounded wait (2^20 polls of its mbarrier) stops its CTA,
 * which waits for that copy once more with a 16 times longer bound, and makes
 * the next lbm_moments / lbm_diagnostics / lbm_get_state on the host return
 * LBM_ERR_CUDA; the lattice's state is then undefined, the context stays
 * usable.  Test hook: the environment variable LBM_TMA_WAIT_POLLS=<n> when
 * staging is set up (lbm_create, lbm_set_tma_staging; lbm_batch_create for a
 * batch) sets the first bound to n polls; n = 0 takes the give-up path at
 * every tile with every copy still completing.  Waits for the handle's
 * stream.  lbm_tma_staging returns 1 or 0. */
int lbm_set_tma_staging(lbm_handle h, int on);
int lbm_tma_staging(lbm_handle h);

/* Replace the handle's stream (borrowed; NULL = legacy default stream). */
int lbm_set_stream(lbm_handle h, void* cuda_stream);

/* The line source of an LBM_BC_CHANNEL lattice (Sec. 4.2): density
 * rho0 + amplitude sin(omega t + phase) at step t, moving at u0 (the paper's
 * omega = 2 per unit time is 2 pi / 100 per step at 200 cells per unit
 * length).  Takes effect from the next call that launches work; waits for
 * the handle's stream.  LBM_ERR_ARG for another boundary or non-finite
 * input. */
int lbm_set_source(lbm_handle h, double amplitude, double omega, double phase);

/* Free the device buffers and the handle.  NULL is allowed. */
void lbm_destroy(lbm_handle h);

/* Device bytes an nx x ny lattice of this storage and boundary holds through
 * its allocator at most: both population buffers, the per-axis absorbing
 * tables, the diagnostics partials, the step counter, the line-source table
 * (LBM_BC_CHANNEL), the TMA error flag (LBM_F32 with LBM_BC_DIRICHLET_EQ) and,
 * with host_io = 1, the FP64 staging of three fields that the first
 * host-memory lbm_init_equilibrium or lbm_moments allocates.  CUDA graphs
 * and tensor maps live outside the allocator and are not counted.  For
 * admission control; 0 for invalid arguments.  No CUDA call. */
size_t lbm_lattice_bytes(int nx, int ny, lbm_storage storage, lbm_bc bc, int host_io);

/* Message of the last non-zero return on h (h = NULL: of the last
 * lbm_create that failed).  Owned by the library. */
const char* lbm_last_error(lbm_handle h);

/* Library version string. */
const char* lbm_version(void);

/* Bandwidth probe for roofline denominators; not part of the scheme.  Copies
 * the `bytes` at device pointer a into b and back, iters times in all, in ONE
 * launch on cuda_stream (a borrowed cudaStream_t, NULL = legacy default):
 * 4 CTAs of 512 threads per SM, each thread owning a fixed, grid-strided set
 * of 16-byte words that it copies in both directions, so no thread waits for
 * another and no launch gap falls between the passes.  Bytes moved = 2 x bytes x
 * iters (read + write).  Asynchronous; time it with events on the stream.
 * LBM_ERR_ARG for NULL or unaligned pointers (16 bytes), bytes not a positive
 * multiple of 16, or iters < 1; LBM_ERR_CUDA if the launch fails. */
int lbm_probe_copy(void* a, void* b, size_t bytes, int iters, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched stepping of many independent lattices (one persistent launch per
 * time step over a tile table, replayed from captured CUDA graphs).
 *
 * Each instance is one problem in the sense of lbm_create + lbm_set_sponge
 * (size, far field, rates, boundary, damping variant, absorbing profile,
 * reference state) plus a step budget.  All instances of a batch share one
 * storage type and one stream.  An instance becomes active at the global step
 * at which it is initialised and stops after exactly its budget of steps, so
 * instances admitted at different times or with different budgets run in the
 * same launches and each takes exactly its own number of steps.  The per-cell
 * arithmetic is that of lbm_step, so a lattice gives the same result alone and
 * in a batch.  Calls on one batch must not overlap from several host threads.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch_ctx* lbm_batch;

/* Device bytes lbm_batch_add allocates for an nx x ny instance (both
 * population buffers and the per-axis absorbing tables), for admission
 * control; 0 for invalid arguments. */
size_t lbm_batch_instance_bytes(int nx, int ny, lbm_storage storage);

/* Create an empty batch on cuda_stream (borrowed) with the given allocator
 * (NULL = cudaMalloc).  Returns LBM_ERR_ARG, LBM_ERR_OOM or LBM_ERR_CUDA on
 * failure. */
int lbm_batch_create(lbm_storage storage, void* cuda_stream, const lbm_allocator* alloc,
                     lbm_batch* out);

/* Tile shape of the batched launch: tile_x in {32, 64, 128, 256} cells along x,
 * tile_y a multiple of 256 / tile_x up to 256 (a block of 256 threads covers
 * the tile in rows).  Default 128 x 8. */
int lbm_batch_set_tiling(lbm_batch b, int tile_x, int tile_y);

/* Cells each thread of the batched launch advances: 1, or 2 (the pair of
 * cells (x, x + 1) on packed FP32 arithmetic, as lbm_set_cells_per_thread;
 * a block of 256 threads then covers tile_x / 2 pairs per row).  2 is the
 * default for LBM_F16DEV and LBM_BF16DEV batches, 1 for LBM_F32 (whose
 * batched step is bound by memory latency, where the one-cell kernel's
 * higher occupancy wins) and LBM_F64 (which has no pair kernel).  The
 * environment variable LBM_CPT=1|2 overrides the default of new batches.
 * LBM_ERR_ARG for any other value or 2 with LBM_F64.  Waits for the batch's
 * stream. */
int lbm_batch_set_cells_per_thread(lbm_batch b, int cells);
/* The current choice (LBM_ERR_ARG for a NULL batch). */
int lbm_batch_cells_per_thread(lbm_batch b);

/* Global time steps per batched launch: 1, or 2 (temporal blocking on tiles
 * of 64 x 16 cells through shared memory, as lbm_set_steps_per_launch; the
 * tile shape of lbm_batch_set_tiling then applies to one-step launches only).
 * An instance whose budget ends after the first step of a two-step launch
 * takes that one step.  Needs two cells per thread
 * (lbm_batch_set_cells_per_thread(b, 1) switches it back to 1).  Default 1.
 * LBM_ERR_ARG for any other value or an unsupported 2.  Waits for the
 * batch's stream. */
int lbm_batch_set_steps_per_launch(lbm_batch b, int steps);
/* The current choice (LBM_ERR_ARG for a NULL batch). */
int lbm_batch_steps_per_launch(lbm_batch b);
/* 1 when the batch's two-step launches stage the input of its Dirichlet
 * instances by TMA (as lbm_set_tma_staging does for one lattice; results
 * bit-identical to plain loads): the default for LBM_F32 batches, chosen at
 * lbm_batch_create (the environment variable LBM_BATCH_TMA=0 keeps plain
 * loads).  A staged copy that times out makes the next lbm_batch_moments /
 * lbm_batch_diagnostics on the host return LBM_ERR_CUDA. */
int lbm_batch_tma_staging(lbm_batch b);

/* Add an instance (arguments as lbm_create and lbm_set_sponge; chi arrays are
 * host arrays, copied) with a budget of nsteps >= 0 steps.  Allocates its
 * buffers; *id receives its handle.  It takes no steps until
 * lbm_batch_init_equilibrium. */
int lbm_batch_add(lbm_batch b, int nx, int ny, double rho0, double ux0, double uy0,
                  const lbm_rates* rates, lbm_bc bc, lbm_variant variant, const double* chi_x,
                  const double* chi_y, double rho_ref, double ux_ref, double uy_ref, int64_t nsteps,
                  int* id);

/* Time 0 of instance id from FP64 fields (as lbm_init_equilibrium); it becomes
 * active from the batch's next step. */
int lbm_batch_init_equilibrium(lbm_batch b, int id, const double* rho, const double* ux,
                               const double* uy, int on_device);

/* Time 0 of instance id as the Gaussian pulse of lbm_init_pulse (built on the
 * device); it becomes active from the batch's next step. */
int lbm_batch_init_pulse(lbm_batch b, int id, double eps, double half_width, double x0,
                         double y0);

/* Advance the batch by nsteps global steps: every active instance takes a step
 * in each of them until its budget is spent.  Asynchronous on the stream. */
int lbm_batch_step(lbm_batch b, int nsteps);

/* Steps instance id has taken (<= its budget), or -1 for an unknown id. */
int64_t lbm_batch_time(lbm_batch b, int id);

/* Fields and diagnostics of instance id at its current time, as lbm_moments
 * and lbm_diagnostics. */
int lbm_batch_moments(lbm_batch b, int id, double* rho_dev, double* ux, double* uy, int on_device);
int lbm_batch_diagnostics(lbm_batch b, int id, int x0, int y0, int x1, int y1, double out[6]);

/* The raw population buffer of instance id at its current time, in the
 * layout of lbm_get_state (bytes = lbm_batch_state_bytes, 0 for an unknown
 * id); on_device selects device or host memory for dst, host transfers
 * synchronise the batch's stream.  LBM_ERR_ARG for an unknown id or a size
 * mismatch, LBM_ERR_STATE before the instance is initialised. */
size_t lbm_batch_state_bytes(lbm_batch b, int id);
int lbm_batch_get_state(lbm_batch b, int id, void* dst, size_t bytes, int on_device);

/* Remove instance id.  Its buffers are released once the launches issued
 * before the call have completed (an event recorded now, checked on later
 * calls and at lbm_batch_destroy); the call itself does not wait. */
int lbm_batch_remove(lbm_batch b, int id);

/* Number of instances in the batch (-1 for NULL). */
int lbm_batch_count(lbm_batch b);

/* Replace the batch's stream (borrowed).  Later calls on the batch issue
 * their work there; work already issued stays where it was.  A caller that
 * moves the batch between streams orders them (events) itself. */
int lbm_batch_set_stream(lbm_batch b, void* cuda_stream);

/* Message of the last error on b. */
const char* lbm_batch_last_error(lbm_batch b);

/* Free every instance and the batch.  NULL is allowed. */
void lbm_batch_destroy(lbm_batch b);

/* ------------------------------------------------------------------------
 * Diagnostics without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory -- for example a host application that owns a fixed device
 * memory pool and forbids other allocations, or a latency-critical loop that
 * cannot afford cudaMalloc/cudaFree (they are slow and may synchronise the
 * whole device).  Such a caller keeps a population buffer of its own (for
 * instance filled by lbm_get_state with on_device = 1) and passes it here.
 *
 * Computes the six sums of lbm_diagnostics over the cells x0 <= ix < x1,
 * y0 <= iy < y1 of `state`: a device buffer in the library's layout for the
 * given storage and lattice (9 planes of ny rows of pitch elements, pitch = nx
 * rounded up to 128 bytes; lbm_state_bytes gives its size), holding the
 * post-collision state that lbm_get_state returns, with far-field state
 * (rho0, u0) and boundary bc.  out: 6 doubles, a device pointer when
 * out_on_device != 0 (the call is then asynchronous on cuda_stream), else a
 * host pointer (the call synchronises cuda_stream).  cuda_stream is a
 * borrowed cudaStream_t (NULL = legacy default stream).
 *
 * Scratch: the block partial sums live in one static device array of
 * 786,480 bytes defined in the library, which every GPU that loads the
 * library holds until the process exits.  The call never calls cudaMalloc,
 * cudaFree or any other allocating routine.  Its first call on a device looks
 * up the array's device address for that device (once per device, with that
 * device current); make that first call before any stream capture.  Every
 * call shares the array and each call rewrites every slot it reads, so no
 * clearing is needed, but calls that overlap on the GPU (on different streams
 * or from several threads) race on it and must be serialised by the caller.
 *
 * Limits: the region may hold at most 268,435,456 cells (16,384 partial sums
 * of 16,384 cells each) and one plane fewer than 2^31 elements; larger inputs
 * return LBM_ERR_TOO_LARGE without touching the device.  Other returns:
 * LBM_ERR_ARG (bad storage; a bc other than LBM_BC_DIRICHLET_EQ or
 * LBM_BC_PERIODIC -- an LBM_BC_CHANNEL state (Sec. 4.2) needs its line source's
 * phase, which this call does not take; bad sizes or region; NULL pointers;
 * rho0 <= 0),
 * LBM_ERR_CUDA, LBM_ERR_NONFINITE (host out only: out is filled and out[5] > 0),
 * LBM_OK. */
#define LBM_ERR_TOO_LARGE (-6) /* input exceeds the fixed capacity of a static scratch */
int lbm_diagnostics_noalloc(const void* state, lbm_storage storage, int nx, int ny, lbm_bc bc,
                            double rho0, double ux0, double uy0, int x0, int y0, int x1, int y1,
                            double* out, int out_on_device, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Von Neumann stability maps (Secs. 3.2-3.3).  These calls need no lattice:
 * they evaluate the scheme linearised about a uniform state f^eq(rho^f, u^f)
 * (the result does not depend on rho^f).  A plane wave of wave vector k is
 * multiplied per step by G(k) = diag(exp(-i k.c_i)) J (Eq. sec:matrix), J the
 * Jacobian of the collision with the damping term of the chosen variant at
 * strength chi (rho* and j* solved exactly, as in the step).
 *
 * A case is LBM_VN_FIELDS consecutive doubles:
 *   s[0..8]  relaxation rates in the row order of M (App. A.1; s[0..2] = s_c),
 *   n, m     Guo weights,  ux_f, uy_f  target velocity u^f,
 *   theta    wave direction,  chi  damping strength (ignored by lbm_vn_chi_crit),
 * and variant[c] is LBM_SPONGE_NONE, _I, _II or _III.  n, m, chi >= 0; every
 * field finite.
 *
 * The growth of a case is max_j max_i |lambda_i(G(k_j))| over
 *   k_j = (pi j / nk)(cos theta, sin theta),  j = 0 .. nk,
 * (the uniform mode and nk wave numbers up to the cut-off pi), computed on
 * the GPU in FP64 (precision = LBM_F64) or FP32 (LBM_F32): Householder
 * reduction to Hessenberg form and the shifted complex QR iteration.
 *
 * Inputs and outputs are HOST arrays; each call copies them, runs on
 * cuda_stream (a borrowed cudaStream_t, NULL = legacy default stream), and
 * synchronises it before returning.  Device scratch is allocated and freed
 * stream-ordered inside the call.
 *
 * Returns LBM_OK; LBM_ERR_ARG (nothing done: bad sizes, NULL arrays, variant,
 * precision, non-finite or negative fields, bad scan parameters);
 * LBM_ERR_OOM; LBM_ERR_CUDA; LBM_ERR_NONFINITE when the QR iteration of some
 * wavenumber did not converge within 270 iterations (that case's output is
 * NaN, the others are valid).  lbm_vn_last_error() gives the message of the
 * last failing call on the calling thread. */
#define LBM_VN_FIELDS 15

/* growth[c] and (if k_at_max != NULL) the |k_j| at which it occurs (the
 * smallest on ties), for c < ncases (0 <= nk <= 2^24). */
int lbm_vn_growth(const int* variant, const double* cases, int ncases, int nk, int precision,
                  double* growth, double* k_at_max, void* cuda_stream);

/* Critical damping strength of each case: chi is scanned on nscan equally
 * spaced values chi_lo .. chi_hi (2 <= nscan <= 4096, 0 <= chi_lo < chi_hi);
 * a value is unstable when growth > 1 + tol.  chi_crit[c] = -INFINITY if
 * chi_lo is already unstable, +INFINITY if no scanned value is, otherwise the
 * midpoint of the interval between the last stable and the first unstable
 * scan value after halving it `iters` times (0 <= iters <= 200).  The smallest
 * unstable chi of Eq. criticalchi is 4/s for type II with equal rates. */
int lbm_vn_chi_crit(const int* variant, const double* cases, int ncases, int nk, int precision,
                    double chi_lo, double chi_hi, int nscan, int iters, double tol,
                    double* chi_crit, void* cuda_stream);

const char* lbm_vn_last_error(void);

/* ------------------------------------------------------------------------
 * Three-dimensional scheme: D3Q15 MRT (transformation matrix of App. A.2)
 * with the damping terms of Secs. 2.2.1-2.2.3, the same definition as the
 * D2Q9 calls above carried to fifteen velocities:
 *   c_i = (0,0,0), (+-1,0,0), (0,+-1,0), (0,0,+-1), then (+-1,+-1,+-1) with x
 *   flipping fastest (rows 1-3 of M); weights 2/9, 1/9, 1/72; c_s^2 = 1/3;
 *   the second-order f^eq and the linear equilibrium w_i (rho + 3 c_i.j).
 * Fields are FP64 [nz][ny][nx] (x fastest), on the host.  Storage: LBM_F64 or
 * LBM_F32 deviations from f^eq(rho0, u0), two buffers of 15 planes of nz x ny
 * rows (pitch = nx rounded up to 128 bytes).  Boundaries: LBM_BC_DIRICHLET_EQ
 * (populations from outside are f^eq(rho0, u0), also at t = 0) or
 * LBM_BC_PERIODIC (all three axes).  Device memory comes from cudaMalloc; the
 * stream is borrowed.  lbm3_step is asynchronous on it; the other calls
 * synchronise it.
 *
 * Returns as above: LBM_OK, LBM_WARN_UNSTABLE_PARAMS (a rate outside (0, 2);
 * chi > 4/s_c for types II/III, s + chi > 2 for type I), LBM_ERR_ARG,
 * LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_STATE. */
typedef struct lbm3_ctx* lbm3_handle;

/* s: 15 rates in the row order of M (s[0..3] = s_c on rho and j).  One plane
 * (pitch * ny * nz elements) must stay below 2^31; ny, nz <= 65535. */
int lbm3_create(int nx, int ny, int nz, lbm_storage storage, double rho0, double ux0, double uy0,
                double uz0, const double* s, double n, double m, lbm_bc bc, void* cuda_stream,
                lbm3_handle* out);
/* Damping variant (LBM_SPONGE_NONE .. LBM_SPONGE_III), per-axis strengths
 * (chi = max of the three at a cell; finite, >= 0) and reference state q_ref. */
int lbm3_set_sponge(lbm3_handle h, lbm_variant variant, const double* chi_x, const double* chi_y,
                    const double* chi_z, double rho_ref, double ux_ref, double uy_ref,
                    double uz_ref);
/* f = f^eq(rho, u) at every cell (time 0). */
int lbm3_init_equilibrium(lbm3_handle h, const double* rho, const double* ux, const double* uy,
                          const double* uz);
int lbm3_step(lbm3_handle h, int nsteps);
/* rho - rho0 and u of the current (streamed, pre-collision) state. */
int lbm3_moments(lbm3_handle h, double* rho_dev, double* ux, double* uy, double* uz);
/* FP64 sums over the cells x0 <= ix < x1, y0 <= iy < y1, z0 <= iz < z1 of the
 * current (streamed) state, in a fixed order (deterministic):
 *   out[0] sum rho'   out[1..3] sum (j - rho0 u0)
 *   out[4] acoustic energy sum [c_s^2 rho'^2 / (2 rho0) + rho0 |u - u0|^2 / 2]
 *   out[5] sum rho'^2   out[6] cells holding a non-finite value.
 * Synchronises the stream.  LBM_ERR_NONFINITE when out[6] > 0 (out filled). */
int lbm3_diagnostics(lbm3_handle h, int x0, int y0, int z0, int x1, int y1, int z1,
                     double out[7]);
/* Checkpoint: the current state buffer (lbm3_state_bytes of them, the layout
 * above) copied to or from HOST memory with its time; synchronises the
 * stream.  lbm3_set_state makes the handle ready to step. */
size_t lbm3_state_bytes(lbm3_handle h);
int lbm3_get_state(lbm3_handle h, void* dst, size_t bytes, int64_t* time);
int lbm3_set_state(lbm3_handle h, const void* src, size_t bytes, int64_t time);
int64_t lbm3_time(lbm3_handle h);
void lbm3_destroy(lbm3_handle h);
/* Message of the handle's last failing call (NULL handle: the calling thread's
 * last lbm3_create failure). */
const char* lbm3_last_error(lbm3_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H_ */
