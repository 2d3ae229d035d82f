/* gks.h -- C ABI of the GB300 compact gas-kinetic scheme library (libgks_gb300.so).
 *
 * The library advances the compact 6th/8th-order gas-kinetic scheme of Zhao, Ji, Shyy
 * and Xu (arXiv:1901.00261) on a uniform 1D or 2D grid:
 *   - per cell it holds the conservative cell averages W = (rho, rho U[, rho V], rho E)
 *     and their cell-averaged gradients W_x [, W_y] (Sec. 1 and Eq. Gausian-formula);
 *   - one step is the two-stage fourth-order MSMD update of Eqs. (step-hyper-1) and
 *     (step-hyper-2), with the interface values updated by the same MSMD (Sec. 2.2);
 *   - interface fluxes, flux time derivatives and interface values come from the
 *     time-accurate gas distribution function of Eq. (3rd-simplify-flux) (Sec. 2.1),
 *     with compact linear reconstruction for the equilibrium part (Sec. 3.1) and compact
 *     WENO-Z for the initial non-equilibrium part (Sec. 3.3); in 2D, three Gauss points
 *     per face and a tangential quartic (Sec. 3.1, last paragraph).
 *
 * Conventions for every call:
 *   - Host state arrays are C-contiguous float64 [nvar][ny][nx], nvar = 3 (1D, ny == 1)
 *     or 4 (2D).  Gradients are dimensional (dW/dx averaged over the cell).
 *   - The caller owns every buffer it passes; the library owns its device buffers
 *     (allocated with cudaMalloc on the current device at gks_create, and at the first
 *     gks_step_host_async for its pipeline slots; freed by gks_destroy).
 *   - Every int-returning call returns GKS_OK (0) or a negative gks_status; the message
 *     of the last error on the calling thread is available from gks_last_error().
 *   - Device work runs on the context's stream (opts.stream, or a stream the library
 *     creates); gks_step_host_async also runs on three streams of its own, ordered with
 *     the context stream by events.  Conditions detected on the device (a non-physical
 *     interface state) are reported by the next synchronising call (gks_get_state*,
 *     gks_sync, gks_max_wavespeed) as GKS_ENONPHYSICAL.
 */
#ifndef GKS_GB300_H
#define GKS_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gks_ctx gks_ctx;

typedef enum gks_status {
  GKS_OK = 0,
  GKS_EINVAL = -1,         /* invalid argument (sizes, order, gamma, dt, NULL pointer) */
  GKS_ECUDA = -2,          /* CUDA runtime error (message in gks_last_error) */
  GKS_ENOMEM = -3,         /* device allocation failed */
  GKS_ENONPHYSICAL = -4,   /* rho <= 0 or p <= 0 met at an interface point */
  GKS_ETIMEOUT = -5        /* reserved: a bounded device wait ran out */
} gks_status;

enum { GKS_RECON_LINEAR = 0, GKS_RECON_WENOZ = 1 };
/* Boundary conditions per axis, applied through two ghost cells per side:
 * GKS_BC_PERIODIC; GKS_BC_TRANSMISSIVE (ghosts copy the boundary cell's W and gradients);
 * GKS_BC_REFLECTING, a solid wall (the reflecting boundary of the blast-wave and
 * double-Mach tests of Sec. 5): ghost k outside the wall is the mirror image of cell k
 * inside, with the momentum normal to the wall negated and, of the gradient normal to the
 * wall, every component but that momentum's negated;
 * GKS_BC_ISOTHERMAL, an isothermal no-slip wall (the walls of the lid-driven cavity of Sec.
 * 5), FP64 form only: ghost k carries the primitive state of cell k inside with the same
 * pressure, the normal velocity negated, the tangential velocity reflected through the
 * wall's (u_t -> 2 u_w - u_t) and the temperature p/rho through the wall's (T -> 2 T_w - T),
 * density p/T, and the derivatives of that ghost field; wall temperatures and velocities in
 * gks_opts.wall_T / wall_u. */
enum { GKS_BC_PERIODIC = 0, GKS_BC_TRANSMISSIVE = 1, GKS_BC_REFLECTING = 2, GKS_BC_ISOTHERMAL = 3 };
/* GKS_PREC_FP64: every step in FP64.
 * GKS_PREC_FP32_BULK: reconstruction, WENO-Z and gas-kinetic arithmetic of the face sweeps in
 * FP32 on differences from a reference cell (the state mirrored as float hi/lo pairs); the
 * time-integration coefficients of the exponential terms and the MSMD accumulation of cell
 * averages in FP64 (conservation is exact); the slopes at the new time level, difference
 * quotients of interface values formed afresh each step, in FP32 (kept in the FP64 state
 * as the exact images of their floats). */
enum { GKS_PREC_FP64 = 0, GKS_PREC_FP32_BULK = 1 };

typedef struct gks_opts {
  double x0, x1, y0, y1;   /* domain; dx = (x1 - x0)/nx, dy = (y1 - y0)/ny */
  int bc_x, bc_y;          /* GKS_BC_PERIODIC, GKS_BC_TRANSMISSIVE, GKS_BC_REFLECTING or
                              GKS_BC_ISOTHERMAL */
  int precision;           /* GKS_PREC_FP64 or GKS_PREC_FP32_BULK */
  double weno_eps;         /* epsilon of the WENO-Z weights, Eq. (WENO-Z-w); default 1e-6 (the
                              paper prints none; 1e-6 reproduces Tables 3-4 of Sec. 4.1) */
  double eps_tau, C_tau;   /* numerical collision time eps*dt + C|pl-pr|/(pl+pr) dt of Sec. 4;
                              defaults 0.01 and 1 */
  int use_graph;           /* 1: replay the two-stage step as a captured CUDA graph */
  int tau_mode;            /* collision time of the Chapman-Enskog terms: 0 (default) mu/p,
                              the physical time; 1 the numerical time above (mu/p, or eps*dt
                              for mu = 0, plus the pressure-jump term of the WENO-Z states),
                              i.e. the same tau in the bracket and the exponentials */
  void* stream;            /* cudaStream_t to run on; NULL: the library creates one */
  int tan_mode;            /* 2D with GKS_RECON_WENOZ, reconstruction along the face (Sec. 3.1,
                              last paragraph): 0 (default) the quartic through five face
                              line-averages for every quantity; 1 the quartic for the
                              equilibrium quantities and five-point WENO-Z at the Gauss points
                              for the initial non-equilibrium states (their values, tangential
                              and normal derivatives), as Sec. 3.3 carried across the face:
                              keeps a discontinuity aligned with the grid physical */
  double wall_T[4];        /* GKS_BC_ISOTHERMAL walls at x0, x1, y0, y1: temperature p/rho
                              (finite, > 0; all four are checked when any wall is isothermal) */
  double wall_u[4];        /* and the wall's velocity along itself (x walls: the y velocity;
                              y walls: the x velocity; unused in 1D).  A moving isothermal
                              wall may not meet a GKS_BC_REFLECTING one (GKS_EINVAL): the
                              mirror image of a moving wall moves the other way */
  int coef_mode;           /* equilibrium Taylor coefficients of Eq. 3rd-simplify-flux (Sec. 2.1):
                              0 (default) the simplified coefficients a_t, a_xt, a_yt, a_tt of
                              the linearised compatibility chain; 1 the full second-order
                              Taylor polynomial of the local Maxwellian (products of the
                              first-order coefficients kept), whose interface values' time
                              derivatives are the Euler equations' own; FP64 form, mu = 0,
                              tau_mode 0 and tan_mode 0 only (GKS_EINVAL otherwise) */
} gks_opts;

/* Fill *o with the defaults: domain [0,1] x [0,1], periodic, FP64, eps 1e-6,
 * eps_tau 0.01, C_tau 1, use_graph 1, tau_mode 0, stream NULL, tan_mode 0, wall_T 1,
 * wall_u 0, coef_mode 0. */
void gks_default_opts(gks_opts* o);

/* Create a solver for nx x ny cells (ny == 1: 1D).  gamma > 1 is the specific-heat ratio
 * of the BGK gas, with K = (4 - 2 gamma)/(gamma - 1) internal degrees of freedom in 2D
 * (Sec. 2.1) and (3 - gamma)/(gamma - 1) in 1D; mu >= 0 the dynamic viscosity, which sets
 * the physical collision time tau = mu/p of Sec. 4 (0: Euler equations); Pr > 0 the
 * Prandtl number (heat flux of the Chapman-Enskog terms scaled by 1/Pr); order 6 or 8, the
 * compact linear reconstruction P^5 or P^7 of Sec. 3.1; recon GKS_RECON_LINEAR or
 * GKS_RECON_WENOZ (compact WENO-Z of Sec. 3.3 for the non-equilibrium states).
 * Requires nx >= 5 and (2D) ny >= 5, every real parameter finite.  opts may be NULL
 * (defaults).  Allocates the device state and work buffers.  Returns NULL on error (see
 * gks_last_error). */
gks_ctx* gks_create(int nx, int ny, double gamma, double mu, double Pr, int order, int recon,
                    const gks_opts* opts);

/* Message of the last error raised on the calling thread ("" if none). */
const char* gks_last_error(void);

/* Copy a host state into the solver: the cell averages W and the cell-averaged gradients
 * Wx, Wy that the compact scheme carries per cell (Sec. 1; they are updated by Eq.
 * Gausian-formula of Sec. 2.2), each [nvar][ny][nx] float64; Wy NULL in 1D.  The caller
 * keeps ownership of the arrays.  Synchronous; GKS_EINVAL for a NULL W or Wx (or Wy in 2D). */
int gks_set_state(gks_ctx* ctx, const double* W, const double* Wx, const double* Wy);

/* Copy the solver state (cell averages and cell-averaged gradients, as gks_set_state) to
 * caller-owned host arrays; synchronises and reports device conditions (GKS_ENONPHYSICAL
 * after a non-physical interface state, the arrays still filled). */
int gks_get_state(gks_ctx* ctx, double* W, double* Wx, double* Wy);

/* Same with device pointers (device-to-device copies, ordered on the context stream;
 * gks_set_state_device returns without synchronising). */
int gks_set_state_device(gks_ctx* ctx, const double* W, const double* Wx, const double* Wy);
int gks_get_state_device(gks_ctx* ctx, double* W, double* Wx, double* Wy);

/* Rows [j0, j0 + nrows) of the 2D state (W, Wx, Wy, each [nvar][ny][nx]) to or from a packed
 * caller-owned device buffer buf laid out [3][nvar][nrows][nx] (W rows, then Wx, then Wy),
 * ordered on the context stream, asynchronous (no host synchronisation): the halo exchange of
 * a row-split decomposition (one problem spread over several GPUs, each holding a slab of
 * rows plus halo rows that its neighbours' steps refresh).  set_rows also refreshes the
 * FP32-bulk form's float mirror of those rows.  GKS_EINVAL for a NULL argument, a 1D context,
 * or rows outside [0, ny). */
int gks_get_rows_device(gks_ctx* ctx, int j0, int nrows, double* buf);
int gks_set_rows_device(gks_ctx* ctx, int j0, int nrows, const double* buf);

/* Advance one two-stage MSMD step of size dt > 0 (asynchronous on the context stream). */
int gks_step(gks_ctx* ctx, double dt);

/* Advance nsteps >= 0 steps of size dt (asynchronous). */
int gks_steps(gks_ctx* ctx, double dt, int nsteps);

/* max over cells of (|U| + c)/dx (+ (|V| + c)/dy in 2D), c = sqrt(gamma p/rho) of the cell
 * averages: the signal speed of the CFL condition of Sec. 4, dt = CFL / *out.  *out is a
 * caller-owned host double.  Synchronises; GKS_ENONPHYSICAL if a cell has rho <= 0 or
 * p <= 0. */
int gks_max_wavespeed(gks_ctx* ctx, double* out);

/* Pipelined step from host memory to host memory, for a stream of independent steps (an
 * ensemble of states, each advanced by one step): copies W, Wx (, Wy) from host memory into
 * one of three device slots, advances that copy one two-stage step of size dt > 0 with the
 * context's scheme, and copies the result into W_out, Wx_out (, Wy_out) in host memory
 * (layout as gks_set_state; Wy and Wy_out NULL in 1D).  Returns without waiting: the copy-in
 * of one call, the step of the call before and the copy-out of the call before that run at
 * the same time (two copy streams beside the context stream), so a run of calls costs about
 * the slowest of the three per call rather than their sum.  The steps run in order with the
 * context's other work; the context's own state is not read or changed.  Every host buffer
 * must stay valid, and the outputs unread, until gks_sync returns; outputs of calls that may
 * be in flight together must not overlap.  Pinned host memory (cudaHostAlloc,
 * cudaHostRegister) gives the overlap; pageable memory works but the copies serialise.  The
 * first call allocates the three slots (three times the state).  Returns GKS_OK,
 * GKS_EINVAL, GKS_ENOMEM or GKS_ECUDA; non-physical states are reported by gks_sync. */
int gks_step_host_async(gks_ctx* ctx, const double* W, const double* Wx, const double* Wy,
                        double* W_out, double* Wx_out, double* Wy_out, double dt);

/* Wait for the context stream and any gks_step_host_async copies; report device
 * conditions. */
int gks_sync(gks_ctx* ctx);

/* Device addresses of the state arrays held by the context (valid until gks_destroy). */
int gks_state_device_ptrs(gks_ctx* ctx, double** W, double** Wx, double** Wy);

/* Number of kernel launches one gks_step issues (for launch accounting). */
int gks_launches_per_step(gks_ctx* ctx);

/* Measurement helpers (not part of the method).
 * gks_steps_timed: advance nsteps steps of size dt with plain launches, each bracketed by
 * CUDA events on the context stream; kernel_ms[k] (k < gks_launches_per_step) receives the
 * summed duration of launch slot k over the steps (slot order: x-face sweep, [y-face sweep,]
 * update, for stage 1 then stage 2).  Synchronises.
 * gks_probe_alu_peak: FLOP/s (FMA = 2) of an FMA-chain kernel over the whole device, in
 * FP64 (fp64 != 0) or FP32; the denominator of the ALU roofline. */
int gks_steps_timed(gks_ctx* ctx, double dt, int nsteps, double* kernel_ms);
int gks_probe_alu_peak(int fp64, double* flops_per_s);
/* Test probe of the non-equilibrium time-integration coefficients (Sec. 2.2: the branch
 * e^{-t/tau} integrated over [0, dt/2] and [0, dt] and fitted linearly in t), evaluated on
 * the device in FP64 exactly as the face kernels form them: for theta[i] = tau/dt > 0
 * (host array, n >= 0 entries), out[4 i + 0..3] (host array) = a0, a1, b0, b1, where with
 * E0(d) = int_0^d e^{-t/tau} dt and E1(d) = int_0^d t e^{-t/tau} dt,
 * a0 = (4 E0(dt/2) - E0(dt))/dt, a1 = (4 E1(dt/2) - E1(dt))/dt,
 * b0 = 4 (E0(dt) - 2 E0(dt/2))/dt^2, b1 = 4 (E1(dt) - 2 E1(dt/2))/dt^2.  Synchronous;
 * GKS_EINVAL for a NULL array, n < 0, dt or a theta not finite and > 0. */
int gks_probe_time_coefs(const double* theta, int n, double dt, double* out);
/* The same coefficients as the single-precision form (GKS_PREC_FP32_BULK) forms them before
 * rounding them to float: FP64 arithmetic, series truncated where the truncation falls below
 * 1e-9 of each coefficient.  Arguments, ownership and errors as gks_probe_time_coefs. */
int gks_probe_time_coefs_single(const double* theta, int n, double dt, double* out);

/* Test probe of the FP64 reciprocal that the single-precision sweeps use for their FP64
 * reference flux (not part of the method): for host x[i] (n >= 0 entries, each positive,
 * normal and within the float range), out[i] (host) = the device's 1/x[i], formed from a
 * single-precision reciprocal refined by two Newton-Raphson steps in FP64.  Synchronous;
 * GKS_EINVAL for a NULL array or n < 0. */
int gks_probe_rcp64(const double* x, int n, double* out);

/* Test probe of the double -> float conversion the FP32-bulk form uses for the float mirror of
 * the slopes (not part of the method): out[i] (host float array) = x[i] (host, n >= 0 entries,
 * any value) rounded to the nearest float, ties to even, as the device forms it on its integer
 * pipes.  Synchronous; GKS_EINVAL for a NULL array or n < 0. */
int gks_probe_d2f(const double* x, int n, float* out);

/* Release everything the context owns.  NULL is ignored. */
void gks_destroy(gks_ctx* ctx);

/* ---- Batches: many independent problems of uneven size, FP32-bulk form ----
 * Every problem is advanced by the same two-stage scheme as gks_step in the FP32-bulk form.
 * One step of the whole batch is one persistent, cooperative kernel launch over a work-list
 * of tiles ordered by phase (stage-1 sweeps, stage-1 updates, stage-2 sweeps, stage-2
 * updates); a tile waits (bounded by a clock budget; GKS_ETIMEOUT if it runs out) until the
 * previous phase of its own problem is complete.  The step is replayed from a CUDA graph.
 * A problem advanced in a batch runs the same arithmetic as when advanced alone with
 * precision GKS_PREC_FP32_BULK; the two agree to single-precision rounding (the compiler
 * fuses multiply-adds differently in the two kernels), not bitwise.  Within a batch the
 * result does not depend on the configuration or on the order tiles are handed out. */
typedef struct gks_batch gks_batch;
typedef struct gks_problem {
  int nx, ny;              /* cells; ny == 1: 1D (nx >= 5; 2D: ny >= 5) */
  int order, recon;        /* 6 | 8; GKS_RECON_LINEAR | GKS_RECON_WENOZ */
  double gamma, mu, Pr;    /* as in gks_create */
  double x0, x1, y0, y1;   /* domain */
  int bc_x, bc_y;          /* GKS_BC_PERIODIC | GKS_BC_TRANSMISSIVE | GKS_BC_REFLECTING (a
                              batch holding a walled problem runs a persistent kernel compiled
                              with the wall signs; isothermal walls: single-problem FP64 form
                              only) */
} gks_problem;

/* Create a batch of n problems (copied); device memory for all of them is one allocation.
 * Returns NULL on error (gks_batch_last_error). */
gks_batch* gks_batch_create(int n, const gks_problem* problems, void* stream);
const char* gks_batch_last_error(void);
/* Host state of problem i ([nvar][ny][nx] float64; Wy NULL in 1D).  Synchronous.
 * set_state also clears problem i's non-physical flag; get_state returns GKS_ENONPHYSICAL
 * (after copying) when problem i has met a non-physical state. */
int gks_batch_set_state(gks_batch* b, int i, const double* W, const double* Wx, const double* Wy);
int gks_batch_get_state(gks_batch* b, int i, double* W, double* Wx, double* Wy);
/* Advance every problem nsteps steps; dt[i] > 0 is problem i's step (asynchronous). */
int gks_batch_steps(gks_batch* b, const double* dt, int nsteps);
int gks_batch_step(gks_batch* b, const double* dt);
/* out[i] = max (|U|+c)/dx (+ (|V|+c)/dy) of problem i.  Synchronises. */
int gks_batch_max_wavespeed(gks_batch* b, double* out);
/* Waits for the batch.  GKS_ETIMEOUT if a dependency wait ran out; GKS_ENONPHYSICAL if any
 * problem met a non-physical interface state (rho <= 0 or p <= 0): such a problem is frozen
 * from that step on (its state is not advanced further and is not meaningful) while every
 * other problem keeps stepping; the message names the problems. */
int gks_batch_sync(gks_batch* b);
/* out[i] (n ints) = GKS_OK or GKS_ENONPHYSICAL for problem i.  Synchronises; returns
 * GKS_ETIMEOUT if a dependency wait ran out. */
int gks_batch_problem_status(gks_batch* b, int* out);
/* Tile shape of the persistent launch: faces (cells) per thread 1, 2 or 4 (2D sweep tiles of
 * 32 x 4, 32 x 8 or 32 x 16 faces; 1D and update items of 128, 256 or 512), and resident
 * blocks per SM (1 .. the occupancy limit of that shape). */
int gks_batch_config(gks_batch* b, int* faces_per_thread, int* blocks_per_sm);
int gks_batch_set_config(gks_batch* b, int faces_per_thread, int blocks_per_sm);
/* Autotuner: time `steps` steps for every tile shape candidate on this batch (the states are
 * restored afterwards), keep the fastest, cache it for batches of the same shape, and write a
 * table of the timings to report (may be NULL). */
int gks_batch_autotune(gks_batch* b, const double* dt, int steps, char* report, int report_len);
/* Clear every status flag (the frozen problems step again) and restore the default wait
 * budget and problem table. */
int gks_batch_reset(gks_batch* b);
/* Test hook for the timeout path: problem `problem`'s items of phase `phase` + 1 will wait for
 * one more producer of phase `phase` than exists, with a wait budget of wait_seconds (<= 10);
 * the next step then ends with every such wait running out and gks_batch_sync returning
 * GKS_ETIMEOUT, with the context still usable (gks_batch_reset restores it). */
int gks_batch_debug_missing_producer(gks_batch* b, int problem, int phase, double wait_seconds);
void gks_batch_destroy(gks_batch* b);

/* ---- One step without any allocation (the paper has no counterpart) ----
 * For callers that cannot call cudaMalloc: code inside a memory pool it does not own, a
 * plug-in whose host forbids device allocation after start-up, or a real-time loop where
 * an allocation and the synchronisation it may bring are not allowed.  Advances one
 * two-stage step of the 1D scheme (same kernels as gks_step) from the caller's device
 * state W, Wx ([3][nx] float64 each) into the caller's device outputs W_out, Wx_out (they
 * may alias the inputs).  All scratch lives in one static device array of the library
 * sized for nx <= GKS_STATIC_MAX_NX cells (about 3.1 MB); every GPU that loads the
 * library holds it until the process exits.  Larger nx is rejected with GKS_EINVAL.
 * The call allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
 * The first call on a device looks up the array's device address on that device; make
 * that first call before any stream capture.  The call itself cannot be captured into a
 * CUDA graph: it synchronises `stream` and reads its status word back to the host.  With lazy module loading
 * (CUDA_MODULE_LOADING=LAZY) the driver places the array in device memory when the
 * library's module is first loaded on a device, which can be that first call: callers that
 * must not allocate after start-up make the first call during start-up.  gamma, mu, Pr,
 * x0, x1 and dt must be finite.  Every call shares the one array and the
 * status word it clears at its start: calls that overlap on the GPU (other streams or
 * threads) race.  Runs on `stream` (NULL: the legacy default stream) and synchronises it
 * before returning; returns GKS_OK, GKS_EINVAL, GKS_ECUDA or GKS_ENONPHYSICAL, with the
 * message in gks_static_last_error().  bc: GKS_BC_PERIODIC, GKS_BC_TRANSMISSIVE or
 * GKS_BC_REFLECTING at both ends. */
#define GKS_STATIC_MAX_NX 16384
int gks_step_1d_static(const double* W, const double* Wx, double* W_out, double* Wx_out,
                       int nx, double gamma, double mu, double Pr, double x0, double x1,
                       int bc, int order, int recon, double dt, void* stream);
const char* gks_static_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GKS_GB300_H */
