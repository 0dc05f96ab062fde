/*
 * lbm.h - C ABI of the GB300 (sm_103a) D2Q9 lattice Boltzmann library.
 *
 * The library implements, as CUDA kernels, the method of Tauzin et al.,
 * "A numerical tool for the study of the hydrodynamic recovery of the
 * Lattice Boltzmann Method" (Comput. & Fluids 172, 2018):
 *   - the D2Q9 BGK time step of eq. (1) with the equilibrium of eq. (2) and
 *     the exact-difference-method forcing named in Sec. 3, on doubly
 *     periodic grids, for a batch ("ensemble") of independent members;
 *   - the sub-volume (L x L box) averages of the energy and enstrophy
 *     balance terms of eqs. (8)-(11), with eq. (17) in time and eq. (18) in
 *     space, and the balancing errors of eqs. (12), (13), for many L;
 *   - an adjoint (reverse-mode) step of the time step and of a box-averaged
 *     dissipation objective (no counterpart in the paper).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: c_0 = (0,0); c_1..c_4 = (1,0), (0,1), (-1,0), (0,-1);
 *          c_5..c_8 = (1,1), (-1,1), (-1,-1), (1,-1); weights 4/9, 1/9, 1/36;
 *          c_s^2 = 1/3.
 * Arrays:  row-major with x fastest.  A scalar field is double[ny][nx]; a
 *          population array is double[9][ny][nx] in the lattice order above.
 * State:   the public state of a member at time n is the pre-collision
 *          population f_l(x, n) of eq. (1).  The device keeps its own
 *          storage convention (post-collision, pull layout, FP32 deviation
 *          g_l = f_l - t_l rho0 for precision 32); the get/set calls convert.
 * Force:   F(x) = F_ext(x) - alpha j(x) with j = sum_l c_l f_l the bare
 *          momentum and F_ext = F0 (sin(2 pi kf y / ny), sin(2 pi kf x / nx))
 *          for force_kind 1 (zero for force_kind 0).  The EDM term is
 *          F_l = f_eq_l(rho, u + F/rho) - f_eq_l(rho, u), u = j / rho.
 * Velocity of the diagnostic: u = (j + F/2) / rho.
 * Memory:  the caller owns every buffer.  The library never allocates device
 *          memory: lbm_workspace_size() states how many bytes of device
 *          memory one handle needs, and the caller passes that buffer to
 *          lbm_create().  Pointers documented as "device" must point into
 *          device memory of the current CUDA device; "host" pointers to
 *          ordinary (ideally pinned) host memory.
 * Streams: all device work of a handle is issued on the stream given in
 *          lbm_config.cuda_stream (NULL = the legacy default stream).  Calls
 *          return once the work is queued, except where a call is documented
 *          as synchronising (it writes host memory).
 * Errors:  every int-returning call returns LBM_OK (0) or a negative
 *          LBM_ERR_* code and never throws; lbm_last_error() gives the
 *          message.  A CUDA error inside a call is reported as LBM_ERR_CUDA.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG (-1)       /* invalid argument */
#define LBM_ERR_WORKSPACE (-2) /* workspace too small or misaligned */
#define LBM_ERR_CUDA (-3)      /* a CUDA call failed */
#define LBM_ERR_HISTORY (-4)   /* fewer than 3 consecutive snapshots */
#define LBM_ERR_DIVERGED (-5)  /* member state contains NaN/Inf or rho <= 0 */
#define LBM_ERR_TIMEOUT (-6)   /* a bounded device wait gave up */

#define LBM_NTERMS 13 /* LHS^E, RHS^{E,1..5}, LHS^Omega, RHS^{Omega,1..6} */
#define LBM_NQUANT 15 /* delta^E, delta^Omega, then the 13 terms */
#define LBM_NGLOBAL 7 /* see lbm_global_balance */

/* One ensemble member: a doubly periodic nx x ny grid (eq. (1)). */
typedef struct lbm_member_cfg {
  int nx, ny;       /* grid size, each >= 1 (the vectorised FP32 kernel
                       serves nx % 4 == 0, another kernel any nx) */
  double tau;       /* BGK relaxation time of eq. (1); nu = (tau - 1/2)/3,
                       eq. (5).  Must be > 0.5 */
  double rho0;      /* reference density of the FP32 deviation storage */
  int force_kind;   /* 0: no external force; 1: Kolmogorov force
                       F0 (sin(2 pi kf y/ny), sin(2 pi kf x/nx));
                       2: the paper's turbulence forcing (Sec. 3): the
                       shell force of eqs. (14), (15) -- streamfunction
                       F0 sum_k cos(2 pi (kx x/nx + ky y/ny) + phase) over
                       one of each pair +-k with 5 <= |k| <= 7, force
                       (d_y psi, -d_x psi) -- plus the large-scale damping
                       of eq. (16): -FR0 times the projection of the bare
                       velocity j/rho of the state being collided on the
                       modes 1 <= |k| <= 2 (one extra read of the
                       populations per step; no adjoint) */
  int kf;           /* Kolmogorov wavenumber, in units of 2 pi / n */
  double F0;        /* Kolmogorov amplitude, or F^T_0 of eq. (14) */
  double alpha;     /* linear drag coefficient on the bare momentum */
  double phase;     /* phi of eq. (14) (force_kind 2) */
  double FR0;       /* F^R_0 of eq. (16) (force_kind 2) */
  int collision;    /* 0: BGK with tau (eq. 1); variable viscosity (Sec. 1)
                       with a local relaxation time from the non-equilibrium
                       stress Pi^neq = -2 rho cs^2 tau S of the pre-collision
                       populations: 1: Smagorinsky nu_t = Cs sqrt(S:S)
                       (S at the local tau itself; closed-form root);
                       2: the turbulent viscosity of eq. (7) (S at tau);
                       3: the entropic LBM (equilibrium minimising
                       H = sum f ln(f/t), relaxation f + alpha (f_eq - f) /
                       (2 tau) with alpha the root of the entropy condition
                       H(f + alpha (f_eq - f)) = H(f), tau_eff = 2 tau /
                       alpha; runs in the general kernel).
                       The diagnostic then uses the local viscosity of each
                       cell at time n; no adjoint */
  double Cs;        /* Smagorinsky constant (collision 1; dx = 1) */
} lbm_member_cfg;

typedef struct lbm_config {
  int n_members;                 /* >= 1 */
  const lbm_member_cfg *members; /* host array of n_members (copied) */
  int precision;   /* 32: FP32 deviation populations; 64: plain FP64 */
  int storage;     /* population storage: 1 = in place (AA pattern: one
                      array, the even step swaps each cell's opposite
                      populations, the odd step reads and writes the
                      neighbours); 2 = double buffer (pull); 0 = chosen by
                      the autotuner at create time together with the launch
                      shape (FP32 ensembles above 1 M cells; otherwise
                      double buffer).  Both move 72 B per FP32 update. */
  int diag_every;  /* > 0: lbm_step records the moment snapshots of the
                      time levels n = k*diag_every - 2, -1, 0 that the
                      eq. (17) time derivative needs; 0: only explicit
                      lbm_record_snapshot() calls record */
  int graph_steps; /* > 0: lbm_step replays CUDA graphs of this many steps
                      (rounded up to even); 0: plain launches */
  int diag_precision; /* arithmetic of the balance terms and box statistics:
                      64 = FP64; 32 = FP32 with every cancelling quantity
                      (time differences, pressure deviation) formed in FP64
                      first; 0 = same as precision.  Snapshots, summed-area
                      tables (exact 64-bit fixed point) and all reductions
                      are exact or FP64 in both cases. */
  int diag_batch;  /* members whose balance diagnostic shares one set of
                      launches (each needs its own scratch slot of about
                      400 B per cell); 0 = as many as fit an 8 GiB budget.
                      Results do not depend on it. */
  void *cuda_stream; /* cudaStream_t of all work; NULL = default stream */
} lbm_config;

typedef struct lbm_handle lbm_handle;

/* Bytes of device workspace a handle with this configuration needs.
 * Host-only; validates the configuration. */
int lbm_workspace_size(const lbm_config *cfg, size_t *bytes);

/* Creates a handle over a caller-owned device workspace (device pointer,
 * 256-byte aligned, at least lbm_workspace_size() bytes, owned by the caller
 * and kept alive until lbm_destroy).  Uploads the member table and the
 * forcing tables; the populations are undefined until lbm_init_fields or
 * lbm_set_populations.  *out receives the handle (host memory owned by the
 * library, freed by lbm_destroy).  Synchronises the stream once. */
int lbm_create(const lbm_config *cfg, void *workspace, size_t bytes,
               lbm_handle **out);

/* Releases the host-side handle and its CUDA graphs; the workspace stays
 * the caller's.  h == NULL is a no-op (returns 0). */
int lbm_destroy(lbm_handle *h);

/* Sets member `member` (or every member when member < 0, all sharing the
 * same fields, which then must fit each member's grid) to the equilibrium
 * state f_l(x, 0) = f_eq_l(rho(x), u(x)) of eq. (2) and resets the step
 * counter and snapshot history of the handle.  rho, ux, uy: double[ny][nx],
 * host pointers if on_device == 0 (pageable memory is copied through the
 * workspace: the call synchronises, and first waits for a queued
 * lbm_subvolume_balance_async, whose scratch it reuses; page-locked memory
 * is read in place like device memory), device pointers otherwise (queued
 * on the stream; an asynchronous diagnostic still running is not waited
 * for: it reads the snapshot ring, not the populations). */
int lbm_init_fields(lbm_handle *h, int member, const double *rho,
                    const double *ux, const double *uy, int on_device);

/* lbm_init_fields for n members at once (the indices in `members`, host
 * array, each listed once, all with the same grid), each from its own
 * fields: rho, ux, uy are double[n][ny][nx] (member members[i] takes block
 * i).  Host pointers (on_device == 0) to pageable memory are copied
 * through the workspace's diagnostic scratch in chunks of whole members,
 * one copy per field and chunk, with a single synchronisation at the end;
 * host pointers to page-locked memory (cudaHostAlloc, cudaHostRegister, a
 * pinned torch tensor; all three fields) and device pointers are read in
 * place by the initialisation kernel, queued on the stream without a
 * synchronisation and without waiting for a queued asynchronous diagnostic
 * (as in lbm_init_fields): the caller keeps page-locked fields unchanged
 * until the stream has passed the call.  With AA storage at an odd step
 * every member must be listed.
 * Resets the step counter and snapshot history like lbm_init_fields. */
int lbm_init_fields_batch(lbm_handle *h, const int *members, int n, const double *rho,
                          const double *ux, const double *uy, int on_device);

/* Advances every member by nsteps time steps of eq. (1): per cell, pull the
 * populations from the neighbours x - c_l, take rho and j, form F, collide
 * with the BGK operator and the EDM term, store.  When diag_every > 0 the
 * snapshots of the required time levels are recorded on the way.  A handle
 * of one member below 32768 cells on the general kernel (without force kind
 * 2) and with graph_steps == 0 runs the consecutive steps between snapshots
 * in one cooperative launch with a grid-wide barrier between steps (same
 * arithmetic, bit-identical results); graph_steps > 0 replays CUDA graphs
 * of per-step launches instead. */
int lbm_step(lbm_handle *h, int nsteps);

/* Current time step n of the handle (number of steps since init). */
long long lbm_time(const lbm_handle *h);

/* Number of CUDA kernels this handle has issued so far (each node of a
 * replayed CUDA graph counts once).  Host-only. */
long long lbm_launch_count(const lbm_handle *h);

/* Launch configuration the handle uses (host-only; any pointer may be NULL):
 * storage 1 (AA) or 2 (double buffer), warps per CTA and rows per warp of
 * the batched FP32 kernel, persistent grid size (0: one CTA per tile), the
 * autotuned time of one step in ms (0 when not tuned), and the rows per
 * thread of the FP32 eq. (16) projection (force kind 2). */
int lbm_tuning(const lbm_handle *h, int *storage, int *warps, int *rows,
               int *grid, float *step_ms, int *proj_rows);

/* Kernels one time step of the handle launches (host-only; -1 for a NULL
 * handle): 1 for the batched FP32 kernel, plus the general kernel's launches
 * for members it does not take, plus the damping projection of eq. (16)
 * when some member has the paper's forcing (force kind 2). */
long long lbm_kernels_per_step(const lbm_handle *h);

/* Sets the launch configuration in place of the autotuned one (host-side;
 * the populations and the storage are kept): for the batched FP32 kernel
 * warps 1..8 per CTA, rows 1, 2 or 4 per warp and grid CTAs (0: one CTA per
 * tile); proj_rows 1..64 rows per thread of the FP32 eq. (16) projection
 * (force kind 2, nx % 4 == 0: a CTA covers 128 x 8 proj_rows cells), 0 to
 * keep the current value.  Results do not depend on any of these.
 * LBM_ERR_ARG for other values, with the previous configuration kept. */
int lbm_set_launch(lbm_handle *h, int warps, int rows, int grid, int proj_rows);

/* Records the moment snapshot (rho, j) of every member at the current time
 * into the 3-slot history used by the eq. (17) time derivative. */
int lbm_record_snapshot(lbm_handle *h);

/* Moments of member `member` at the current time (device pointers,
 * double[ny][nx] each, any may be NULL): rho = sum f (below eq. (2)),
 * u = (j + F/2)/rho, and the vorticity omega = D_x u_y - D_y u_x with D the
 * 8th-order centred difference of eq. (18). */
int lbm_moments(lbm_handle *h, int member, double *rho, double *ux,
                double *uy, double *omega);

/* Whole-grid quantities of member `member` at the current time, in FP64
 * (host pointer to LBM_NGLOBAL doubles; synchronises):
 *   out[0] = sum rho, out[1] = sum j_x, out[2] = sum j_y,
 *   out[3] = <E> = mean of rho |u|^2 / 2, out[4] = <Omega> = mean of w^2/2,
 *   out[5] = <u . F>, out[6] = <eps> = mean of nu rho S_ij d_j u_i
 * (u the diagnostic velocity, S_ij = d_j u_i + d_i u_j, eq. (18) stencils):
 * the L = N case of the energy/enstrophy budget of eqs. (8)-(11). */
int lbm_global_balance(lbm_handle *h, int member, double *out);

/* Sub-volume balance of member `member` at the current time n (eqs. (8)-(13),
 * (17), (18)), for each box size L[i] (i < nL; host array):
 * the local terms LHS^E, RHS^{E,1..5}, LHS^Omega, RHS^{Omega,1..6} are
 * formed from the snapshots at n, n-1, n-2 (the snapshot at n is recorded
 * if missing; LBM_ERR_HISTORY if n-1 or n-2 is missing), averaged over L x L
 * boxes (periodic wrap) through exact fixed-point summed-area tables, and
 * turned into the balancing errors delta^E, delta^Omega (0 when numerator
 * and denominator are 0, +Inf when only the denominator is).
 * Boxes: with origins == NULL and counts == NULL, every one of the nx*ny
 * periodic origins for every L; otherwise counts[i] (host, >= 1) boxes for
 * L[i], whose lower-left corners (x0, y0) are the host pairs of origins
 * (0 <= x0 < nx, 0 <= y0 < ny), concatenated in the order of L (e.g. the
 * paper's Table 1 random boxes).
 * Sizes with L < 1 or L > min(nx, ny) are skipped: their statistics are NaN.
 * stats_out (host, double[nL][15][2]; synchronises): mean and population
 * standard deviation over the boxes of the 15 quantities
 * [delta^E, delta^Omega, LHS^E, RHS^{E,1..5}, LHS^O, RHS^{O,1..6}].
 * per_box_out (device, may be NULL; then every L must fit the grid, else
 * LBM_ERR_ARG): double[rows][15], one row per box in the order of L (nL * nx
 * * ny rows for all origins, sum(counts) rows for lists). */
int lbm_subvolume_balance(lbm_handle *h, int member, const int *L, int nL,
                          const int *origins, const int *counts,
                          double *stats_out, double *per_box_out);

/* The same diagnostic for the n_members members listed in the host array
 * members[], queued back to back with a single synchronisation at the end:
 * stats_out (host) is double[n_members][nL][15][2], each member's sizes
 * checked against its own grid.  origins and counts, when given, apply to
 * every member.  No per-box output. */
int lbm_subvolume_balance_batch(lbm_handle *h, const int *members,
                                int n_members, const int *L, int nL,
                                const int *origins, const int *counts,
                                double *stats_out);

/* Largest number of histogram bin edges per quantity. */
#define LBM_MAX_EDGES 256

/* Distributions over the boxes of each size, for the members listed in the
 * host array members[] (boxes, sizes and the synchronisation as
 * lbm_subvolume_balance_batch): the histograms behind the paper's PDFs of
 * the balancing errors (Sec. 4, at fixed l = L / N) and the sub-volume Mach
 * number of eq. (20), read as Ma_V = sqrt(<u_x^2 + u_y^2>_V) / c_s with the
 * diagnostic velocity u.
 * delta_edges (host, n_delta_edges in 1..LBM_MAX_EDGES) and mach_edges
 * (host, n_mach_edges): finite, strictly ascending bin edges e_0 < e_1 < ...;
 * a value v goes to bin b = the number of edges <= v (bin 0: v < e_0; the
 * last bin: v >= e_last, +Inf included; NaN in no bin).
 * stats_out (host, may be NULL): the statistics of
 * lbm_subvolume_balance_batch, double[n_members][nL][15][2].
 * delta_hist_out (host): long long[n_members][nL][2][n_delta_edges + 1],
 *   box counts of delta^E (index 0) and delta^Omega (1) per bin;
 * mach_hist_out (host): long long[n_members][nL][n_mach_edges + 1];
 * mach_stats_out (host): double[n_members][nL][2], mean and population
 *   standard deviation of Ma_V over the boxes.
 * Sizes that do not fit a member give zero counts and NaN statistics.
 * Counts are exact integers (independent of launch order); the bin of a
 * value is decided in the diagnostic precision (FP32 or FP64), so a value
 * within rounding of an edge may fall on either side of it relative to an
 * FP64 evaluation.  LBM_ERR_ARG for invalid edges or NULL outputs. */
int lbm_subvolume_distributions(lbm_handle *h, const int *members,
                                int n_members, const int *L, int nL,
                                const int *origins, const int *counts,
                                const double *delta_edges, int n_delta_edges,
                                const double *mach_edges, int n_mach_edges,
                                double *stats_out, long long *delta_hist_out,
                                long long *mach_hist_out,
                                double *mach_stats_out);

/* Asynchronous form of lbm_subvolume_balance_batch: the diagnostic of the
 * current time is queued on an internal stream after the work already queued
 * on the handle's stream (its snapshots), and the call returns without
 * waiting.  stats_dev (device, double[n_members][nL][15][2], NaN for skipped
 * sizes) receives the statistics; it and the host arrays may be reused once
 * lbm_diag_synchronize has returned (the host arrays right away).  Later
 * calls that need the snapshot ring or the diagnostic scratch (the next
 * snapshot record, moments, balances, adjoint, host transfers) are ordered
 * after it on the device, so the stepping of the next diagnostic period runs
 * concurrently with it. */
int lbm_subvolume_balance_async(lbm_handle *h, const int *members,
                                int n_members, const int *L, int nL,
                                const int *origins, const int *counts,
                                double *stats_dev);

/* Blocks the host until the last asynchronous diagnostic has finished. */
int lbm_diag_synchronize(lbm_handle *h);

/* Public pre-collision populations f_l(x, n) of member `member` as
 * double[9][ny][nx] (full f, also for FP32 storage).  Host pointer if
 * on_device == 0 (the call synchronises), device pointer otherwise.
 * get then set restores the FP64 state bit for bit. */
int lbm_get_populations(lbm_handle *h, int member, double *f, int on_device);
int lbm_set_populations(lbm_handle *h, int member, const double *f,
                        int on_device);

/* Divergence check of member `member` at the current time: *status = 1 if
 * any population or density is NaN/Inf or rho <= 0, else 0.  Synchronises.
 * Returns LBM_ERR_TIMEOUT if a step of a small single-member handle (which
 * runs all the steps of an lbm_step call in one cooperative launch with a
 * grid-wide barrier between steps) gave up waiting at that barrier. */
int lbm_member_status(lbm_handle *h, int member, int *status);

/* Adjoint of one time step of member `member` (no counterpart in the paper;
 * the differentiation of the forward model).  With the forward map
 * f(n+1) = S(f(n); tau, F0) of eq. (1), given lambda_in = dJ/df(n+1) as
 * double[9][ny][nx] (device), writes lambda_out = (dS/df(n))^T lambda_in
 * + dJ_n/df(n) (device, may not alias lambda_in), where J_n is the
 * objective term at time n: the L x L box average, origin (bx, by), of the
 * dissipation term RHS^{E,4} of eq. (8), weighted by obj_weight (0 to omit).
 * f_n (device, double[9][ny][nx]) is the public state at time n.  The
 * contributions of this step to dJ/dtau and dJ/dF0 are ADDED to the FP64
 * accumulators at the device pointers dJ_dtau and dJ_dF0.  Plain FP64
 * (either handle precision). */
int lbm_adjoint_step(lbm_handle *h, int member, const double *f_n,
                     const double *lambda_in, double *lambda_out,
                     double obj_weight, int bx, int by, int L,
                     double *dJ_dtau, double *dJ_dF0);

/* acc[0] += weight * (L x L box average, origin (bx, by), of the dissipation
 * term RHS^{E,4} of eq. (8) of member `member` at the current time): the
 * forward objective matching lbm_adjoint_step.  acc is a device pointer to
 * one double.  One kernel launch (the moments of the box widened by the
 * 4-cell reach of the eq. (18) stencils only, per tile of the box, and a
 * fixed-order sum: the result does not depend on the launch order). */
int lbm_objective_accumulate(lbm_handle *h, int member, double weight, int bx,
                             int by, int L, double *acc);

/* The same objective at nsteps consecutive time levels: acc[0] += weight *
 * (box average at the current time), then one step of every member, nsteps
 * times, so the handle ends nsteps steps later.  One call replaces nsteps
 * pairs of lbm_objective_accumulate and lbm_step(h, 1). */
int lbm_objective_steps(lbm_handle *h, int member, int nsteps, double weight,
                        int bx, int by, int L, double *acc);

/* Public states of member `member` at nstates consecutive times: states[k]
 * (device, double[nstates][9][ny][nx]) receives f(t + k) for the current
 * time t and k = 0 .. nstates - 1, stepping every member nstates - 1 times
 * in between (the recomputation of a checkpoint interval for the adjoint).
 * The handle ends at time t + nstates - 1. */
int lbm_record_trajectory(lbm_handle *h, int member, int nstates,
                          double *states);

/* lbm_adjoint_step over nstates consecutive time levels, last to first:
 * states[k] (device, double[nstates][9][ny][nx]) is the public state
 * f(n + k), lambda_in = dJ/df(n + nstates) (device; NULL for zero) and, for
 * k = nstates - 1 down to 0, lambda(n + k) = (dS/df)^T lambda(n + k + 1)
 * + weights[k] * dJ_{n+k}/df, the objective term as in lbm_adjoint_step
 * with weights a host array of nstates doubles (0 omits a level).  The
 * result lambda(n) is written to lambda_out; lambda_tmp (device, same size)
 * is the other half of the ping-pong; lambda_in, lambda_out and lambda_tmp
 * must be three distinct buffers.  dJ/dtau and dJ/dF0 contributions are
 * added to the device accumulators as in lbm_adjoint_step, summed over the
 * whole call before they are added (one reduction per call: the adjoint
 * fields equal those of nstates lbm_adjoint_step calls bit for bit, the two
 * gradients up to the order of their FP64 sums).  Non-finite weights, or a
 * box outside the grid when some weight is non-zero, return LBM_ERR_ARG
 * before any work. */
int lbm_adjoint_sweep(lbm_handle *h, int member, const double *states,
                      int nstates, const double *lambda_in, double *lambda_out,
                      double *lambda_tmp, const double *weights, int bx, int by,
                      int L, double *dJ_dtau, double *dJ_dF0);

/* Measured arithmetic ceiling (no counterpart in the paper; a measurement
 * helper): FP64 (bits = 64) or FP32 (bits = 32) fused multiply-adds of
 * independent chains on every SM, timed with CUDA events on cuda_stream
 * (NULL = legacy default stream); *flops_per_s (host) receives the rate,
 * two flops per FMA.  Synchronises the stream; about 20 ms. */
int lbm_probe_fma_rate(int bits, void *cuda_stream, double *flops_per_s);

/* The grid-wide barrier of the small-grid persistent step, alone (no
 * counterpart in the paper; for testing its failure detection): `rounds`
 * barriers over `ctas` cooperative 32-thread CTAs (ctas no more than can be
 * co-resident, else LBM_ERR_CUDA).  If withhold >= 0, CTA `withhold` never
 * arrives: the others give up after their bounded wait (a second at most)
 * and set the error word, which *gave_up (host) receives (1), without any
 * device fault.  Synchronises cuda_stream. */
int lbm_probe_grid_barrier(int ctas, int rounds, int withhold, void *cuda_stream,
                           int *gave_up);

/* Largest grid (nx * ny cells) that lbm_global_balance_static accepts. */
#define LBM_STATIC_MAX_CELLS (512 * 512)

/* Allocation-free variant of lbm_global_balance (the paper has no
 * counterpart; this is an interface of this library).
 *
 * For callers that cannot allocate device memory: for example a plug-in
 * whose host application owns the whole device memory pool, or code that
 * must not call cudaMalloc because it implicitly synchronises the device.
 * Such callers cannot provide the workspace that lbm_create needs, so this
 * entry point takes no handle: it computes the same 7 quantities as
 * lbm_global_balance (same order, FP64) directly from caller-owned
 * populations, using a fixed scratch array that the library holds in
 * device memory (about 4.3 MB on every GPU that loads the library, until the
 * process exits).
 *
 * f:   device pointer, double[9][ny][nx], the public pre-collision
 *      populations f_l(x, n) (as written by lbm_get_populations).
 * nx, ny: grid, 1 <= nx * ny <= LBM_STATIC_MAX_CELLS (larger grids return
 *      LBM_ERR_ARG with a message; use lbm_global_balance for them).
 * m:   host pointer to the member parameters (tau, force_kind, kf, F0,
 *      alpha are used; rho0 is not); force kinds 0 and 1 with the BGK
 *      collision only (others return LBM_ERR_ARG).
 * out: host pointer to LBM_NGLOBAL doubles; the call synchronises
 *      cuda_stream (NULL = legacy default stream) before returning.
 * m->tau must be finite and above 1/2, F0 and alpha finite.
 * Calls no cudaMalloc or cudaFree.  The first call on a device looks up the
 * scratch address with cudaGetSymbolAddress; make that first call before
 * any stream capture.  The address is kept for the rest of the process:
 * resetting the device (cudaDeviceReset) after that first call is not
 * supported.  Every call on a device shares the one scratch array
 * (which keeps the last call's contents): calls whose work overlaps on the
 * GPU, e.g. on two streams at once, race and give wrong results.  Errors are
 * reported through lbm_static_last_error(). */
int lbm_global_balance_static(const double *f, int nx, int ny,
                              const lbm_member_cfg *m, double *out,
                              void *cuda_stream);

/* Message of the last failing lbm_global_balance_static call of this host
 * thread.  Never NULL. */
const char *lbm_static_last_error(void);

/* Message of the last failing call on this handle (or of the last failing
 * handle-less call when h is NULL).  Never NULL. */
const char *lbm_last_error(const lbm_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H_ */
