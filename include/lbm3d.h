/*
 * Three-dimensional extension of the GB300 library (liblbm.so): the D3Q19
 * and D3Q27 lattice BGK of eq. (1) with the eq. (2) equilibrium and exact-difference
 * forcing (Sec. 3) of Tauzin et al. (2018), and the sub-volume energy and
 * enstrophy balance of eqs. (8)-(13) in their general index forms, where
 * the vortex-stretching term RHS^{Omega,6} = omega_i omega_j d_j u_i does
 * not vanish (the paper's outlook).  Same conventions as lbm.h: the caller
 * owns all memory, work is queued on cfg->cuda_stream, errors are negative
 * LBM_ERR_* codes (lbm.h) with a message from lbm3d_last_error.
 *
 * Lattice order: c_0 = 0; c_1..6 = +x, -x, +y, -y, +z, -z; c_7..18 =
 * (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1),
 * (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1): D3Q19, weights 1/3,
 * 1/18, 1/36.  D3Q27 adds the corners c_19..26 = (1,1,1), (-1,-1,-1),
 * (1,1,-1), (-1,-1,1), (1,-1,1), (-1,1,-1), (-1,1,1), (1,-1,-1), weights
 * 8/27, 2/27, 1/54, 1/216 by |c|^2 = 0..3; both with c_s^2 = 1/3 and the
 * eq. (2) equilibrium.  Public populations: double[q][nz][ny][nx] (x
 * fastest, q = 19 or 27), the pre-collision f_l(x, n) of eq. (1); fields
 * double[nz][ny][nx].
 */
#ifndef LBM3D_H
#define LBM3D_H

#include <stddef.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3d_member_cfg {
  int nx, ny, nz;   /* grid, each >= 1 */
  double tau;       /* relaxation time of eq. (1), > 0.5; nu = (tau - 1/2)/3 */
  double rho0;      /* reference density of the FP32 deviation storage */
  int force_kind;   /* 0: none; 1: cyclic Kolmogorov force F0 (sin(2 pi kf
                       y/ny), sin(2 pi kf z/nz), sin(2 pi kf x/nx)) */
  int kf;           /* Kolmogorov wavenumber in units of 2 pi / n */
  double F0;        /* Kolmogorov amplitude */
  double alpha;     /* linear drag on the bare momentum: F = F_ext - alpha j */
} lbm3d_member_cfg;

typedef struct lbm3d_config {
  int n_members;                    /* >= 1 */
  const lbm3d_member_cfg *members;  /* host array (copied) */
  int precision;    /* 32: FP32 deviations f - t rho0; 64: FP64 */
  int diag_every;   /* > 0: lbm3d_step records the snapshots of the times
                       k diag_every - 2, -1, 0 that eq. (17) needs */
  void *cuda_stream; /* cudaStream_t of all work; NULL = default stream */
  int lattice;      /* velocity set of every member: 19 (D3Q19; also 0) or 27
                       (D3Q27); anything else is LBM_ERR_ARG */
  int diag_precision; /* arithmetic of the balance terms: 64 (also 0) FP64;
                         32 FP32 (level differences formed in FP64 from the
                         FP64 snapshots, rounded once) */
} lbm3d_config;

typedef struct lbm3d_handle lbm3d_handle;

/* Device workspace bytes for a configuration (host-only; validates it). */
int lbm3d_workspace_size(const lbm3d_config *cfg, size_t *bytes);

/* Carves every device buffer out of `workspace` (device, 256-byte aligned,
 * >= lbm3d_workspace_size bytes, owned by the caller and kept alive until
 * lbm3d_destroy).  *out receives the handle. */
int lbm3d_create(const lbm3d_config *cfg, void *workspace, size_t bytes, lbm3d_handle **out);
/* Waits for the handle's work and releases it (host memory; the workspace
 * stays the caller's).  h == NULL is a no-op (returns 0). */
int lbm3d_destroy(lbm3d_handle *h);

/* f(x, 0) = f_eq(rho(x), u(x)) (eq. 2) for one member; rho, ux, uy, uz are
 * double[nz][ny][nx], host (on_device = 0) or device pointers. */
int lbm3d_init_fields(lbm3d_handle *h, int member, const double *rho, const double *ux,
                      const double *uy, const double *uz, int on_device);

/* nsteps steps of eq. (1) for every member: one launch per step for the FP32
 * members with nx % 4 == 0, one per member and step for the others. */
int lbm3d_step(lbm3d_handle *h, int nsteps);
long long lbm3d_time(const lbm3d_handle *h);
/* Cells per lane of the vectorised FP32 kernel that every FP32 member with
 * nx % 4 == 0 takes: 4 or 2, the faster on this device, timed at create time
 * for ensembles above 1 M cells (4 otherwise); 0 when no member takes it; -1
 * for a NULL handle.  Host-only.  Results do not depend on it. */
int lbm3d_cells_per_lane(const lbm3d_handle *h);
/* Sets the cells per lane of that kernel (4 or 2; LBM_ERR_ARG otherwise, the
 * setting kept).  Host-side: the populations are kept. */
int lbm3d_set_cells_per_lane(lbm3d_handle *h, int cpl);

/* Public populations double[q][nz][ny][nx] of one member, host or device
 * (index for index the oracle's f(., n)); set accepts the same layout. */
int lbm3d_get_populations(lbm3d_handle *h, int member, double *f, int on_device);
int lbm3d_set_populations(lbm3d_handle *h, int member, const double *f, int on_device);

/* Records the (rho, j) snapshot of the current time (also done by
 * lbm3d_step at the times diag_every requests). */
int lbm3d_record_snapshot(lbm3d_handle *h);

/* Sub-volume balance of one member at the current time n (snapshots of n,
 * n-1, n-2 required; LBM_ERR_HISTORY otherwise): the 13 local terms in FP64
 * (eq. (18) in space, eq. (17) in time), L x L x L box averages with
 * periodic wrap through exact 64-bit fixed-point summed-volume tables,
 * delta^E and delta^Omega (eqs. (12), (13); the enstrophy balance with its
 * six right-hand terms), and per size the mean and population standard
 * deviation of [delta^E, delta^Omega, LHS^E, RHS^{E,1..5}, LHS^O,
 * RHS^{O,1..6}] into stats_out (host, double[nL][15][2]; synchronises).
 * Boxes: every periodic origin (origins == counts == NULL) or counts[i]
 * lower corners for L[i] given as host int triples (x0, y0, z0) in
 * `origins`, concatenated in the order of L.  Sizes above min(nx, ny, nz)
 * give NaN.  per_box_out (device, nullable; every size must fit): double
 * [rows][15], one row per box in the order of L. */
int lbm3d_subvolume_balance(lbm3d_handle *h, int member, const int *L, int nL,
                            const int *origins, const int *counts, double *stats_out,
                            double *per_box_out);

const char *lbm3d_last_error(const lbm3d_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* LBM3D_H */
