// Internal definitions of the GB300 D2Q9 library: member table, storage
// layout and device helpers shared by the kernels of this library.
//
// Storage convention (device): for member m, buffer b in {0, 1},
//   pop[b][(l * ny + y) * pitch + x]   (SoA planes, x fastest, pitch >= nx)
// holds the post-collision population f*_l at its ORIGIN cell x (pull
// layout), so that the pre-collision population of eq. (1) at time n is
//   f_l(x, n) = pop[cur][l][x - c_l]   (periodic).
// Precision 32 stores the deviation g_l = f_l - t_l rho0 (float); precision
// 64 stores f_l itself (double).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr int kQ = 9;
// D2Q9 velocities and weights (order: rest, 4 axis, 4 diagonal).
__host__ __device__ constexpr int cx_of(int l) {
  return l == 1 || l == 5 || l == 8 ? 1 : (l == 3 || l == 6 || l == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int l) {
  return l == 2 || l == 5 || l == 6 ? 1 : (l == 4 || l == 7 || l == 8 ? -1 : 0);
}
__host__ __device__ constexpr double w_of(int l) {
  return l == 0 ? 4.0 / 9.0 : (l <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr int opposite(int l) {
  return l == 0 ? 0 : (l <= 4 ? ((l + 1) % 4) + 1 : ((l - 5 + 2) % 4) + 5);
}

// Per-member parameters, uploaded once into the workspace.
struct Member {
  int nx, ny, pitch;     // grid and row pitch (elements)
  int force_kind, kf;
  int pad0;
  double tau, omega;     // omega = 1 / tau
  double rho0, F0, alpha;
  float rho0_f, omega_f, alpha_f;  // float copies for the FP32 kernels
  int pad1;
  double nu;             // (tau - 1/2) / 3
  size_t plane;          // ny * pitch
  void *pop[2];          // population buffers
  void *fx_tab;          // F_ext,x as function of y: [ny] (float or double)
  void *fy_tab;          // F_ext,y as function of x: [nx]
  double *fx_tab64;      // the same tables in double (diagnostics, adjoint)
  double *fy_tab64;
  double *snap;          // ring of 3 slots of (rho, jx, jy), 24 B per cell each:
                         // FP64 [3][N], or FP32 storage (hi, lo) pairs
                         // [3][2][N] of rho - rho0, jx, jy
  int *status;           // divergence flag
  // force kind 2 (shell force of eqs. (14), (15), damping of eq. (16))
  double FR0;
  void *ft_tab;          // shell force F^T: [2][ny][pitch] (float or double)
  double *ft_tab64;      // the same in FP64, [2][ny * nx]
  void *trig;            // cos, sin of 2 pi x/nx and 4 pi x/nx ([4][nx]), then
                         // of 2 pi y/ny and 4 pi y/ny ([4][ny]) (float or double)
  double *trig64;        // the same in FP64
  double *damp;          // damping coefficients of the state being stepped
  float *damp_f;         // (kDamp values, layout at damping_at) and float copies
  double *damp_ring;     // the coefficients of each snapshot ring slot [3][kDamp]
  double *proj_part;     // projection CTA partials [CTAs][kDamp]
  float *damp_rows;      // FP32 storage: per-row damping factors [ny][6]
  unsigned *proj_count;  // CTAs of the projection done (zero between launches)
  // variable-viscosity collision (1: Smagorinsky, 2: eq. (7)); 0: BGK
  int collision;
  float Cs_f, tau_f;     // float copies of Cs and tau
  double Cs;
  void *nu_ring;         // local viscosity at each snapshot slot [3][N]
                         // (storage precision), collision != 0
};

// Local relaxation time of a cell from its non-equilibrium stress
// Pi^neq = sum c c (f - f_eq), f_eq of eq. (2) at u = j / rho, through the
// Chapman-Enskog relation Pi^neq = -2 rho cs^2 tau S:
//   1: Smagorinsky nu_t = Cs sqrt(S:S) with S at the local tau itself, the
//      positive root tau = (tau0 + sqrt(tau0^2 + 18 Cs |Pi| / rho)) / 2;
//   2: eq. (7), nu_t = -(cs^2 / 3) tau0^2 Tr(S^3) / Tr(S^2) with S at tau0,
//      tau = tau0 + tau0 Tr(Pi^3) / (2 rho Tr(Pi^2)).
// pxx, pxy, pyy: the components of Pi^neq; rho the density.
template <typename T>
__host__ __device__ inline T tau_from_stress(T pxx, T pxy, T pyy, T rho, T tau0, int coll,
                                             T Cs) {
  const T tr2 = pxx * pxx + T(2) * pxy * pxy + pyy * pyy;
  if (coll == 1) return T(0.5) * (tau0 + sqrt(tau0 * tau0 + T(18) * Cs * sqrt(tr2) / rho));
  if (tr2 == T(0)) return tau0;
  const T a2xx = pxx * pxx + pxy * pxy, a2xy = pxy * (pxx + pyy), a2yy = pxy * pxy + pyy * pyy;
  const T tr3 = a2xx * pxx + T(2) * a2xy * pxy + a2yy * pyy;
  return tau0 + tau0 * tr3 / (T(2) * rho * tr2);
}

// Damping coefficients of eq. (16): for component c (0: x, 1: y) and the
// representatives m of the 6 pairs +-k, 1 <= |k| <= 2, in the order (1,0),
// (0,1), (1,1), (1,-1), (2,0), (0,2): A = -2 F^R_0 C, B = -2 F^R_0 S at
// [c * 12 + 2 m] and [c * 12 + 2 m + 1], with C, S the means over the grid
// of u_c cos(theta_m), u_c sin(theta_m).  The pair sums double the terms.
constexpr int kDamp = 24;

// F^R(x, y) from the coefficients D and the trig tables (layout at
// Member::trig): sum_m A_m cos(theta_m) + B_m sin(theta_m), with the (1,1)
// and (1,-1) terms regrouped by the angle-sum identities.
template <typename T, typename C>
__host__ __device__ inline void damping_at(const C *D, const T *trig, int nx, int ny, int x,
                                           int y, T &fx, T &fy) {
  const T cx = trig[x], sx = trig[nx + x], c2x = trig[2 * nx + x], s2x = trig[3 * nx + x];
  const T *ty = trig + 4 * nx;
  const T cy = ty[y], sy = ty[ny + y], c2y = ty[2 * ny + y], s2y = ty[3 * ny + y];
  T out[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const C *d = D + 12 * k;
    const T A0 = (T)d[0], B0 = (T)d[1], A1 = (T)d[2], B1 = (T)d[3], A2 = (T)d[4], B2 = (T)d[5];
    const T A3 = (T)d[6], B3 = (T)d[7], A4 = (T)d[8], B4 = (T)d[9], A5 = (T)d[10], B5 = (T)d[11];
    const T P = A0 + (A2 + A3) * cy + (B2 - B3) * sy;
    const T Q = B0 + (B2 + B3) * cy - (A2 - A3) * sy;
    const T R = A1 * cy + B1 * sy + A5 * c2y + B5 * s2y;
    out[k] = P * cx + Q * sx + A4 * c2x + B4 * s2x + R;
  }
  fx = out[0];
  fy = out[1];
}

// Tile of the batched stream-collide: member, first x, first y.
struct Tile {
  int member, x0, y0, pad;
};

#ifdef __CUDACC__
// One-cell periodic shift.
__device__ __forceinline__ int wrap1(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Storage index of the public population f_l(x, y) in a given state.
__device__ __forceinline__ size_t pub_index(const Member &M, int state, int l, int x, int y) {
  if (state == 2) return (size_t)l * M.plane + (size_t)y * M.pitch + x;
  const int xs = wrap1(x - cx_of(l), M.nx), ys = wrap1(y - cy_of(l), M.ny);
  const int slot = state == 3 ? opposite(l) : l;
  return (size_t)slot * M.plane + (size_t)ys * M.pitch + xs;
}
__device__ __forceinline__ void *state_buffer(const Member &M, int state) {
  return state < 2 ? M.pop[state] : M.pop[0];
}

// Error-free addition (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Compensated FP32 sum of FP32 values, returned in FP64: the value of a
// double-precision sum at FP32 arithmetic cost (GB300 runs FP64 at a small
// fraction of its FP32 rate).
__device__ __forceinline__ double csum(const float *v, const int *sign, int n) {
  float s = sign[0] * v[0], c = 0.f;
  for (int k = 1; k < n; ++k) {
    float e;
    two_sum(s, sign[k] * v[k], s, e);
    c += e;
  }
  return (double)s + (double)c;
}

// (rho, j_x, j_y) in FP64 of one cell's public populations: FP32 deviations
// g = f - t rho0 by compensated sums (rho = rho0 + sum g: the weights sum to
// 1), FP64 populations by plain sums in index order.
template <typename T>
__device__ __forceinline__ void pub_moments(const T (&f)[kQ], double rho0, double &r, double &jx,
                                            double &jy) {
  if constexpr (sizeof(T) == 4) {
    const int one[kQ] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    const float ax[6] = {f[1], f[5], f[8], f[3], f[6], f[7]};
    const float ay[6] = {f[2], f[5], f[6], f[4], f[7], f[8]};
    const int sgn[6] = {1, 1, 1, -1, -1, -1};
    r = rho0 + csum(f, one, kQ);
    jx = csum(ax, sgn, 6);
    jy = csum(ay, sgn, 6);
  } else {
    r = 0.0;
    jx = 0.0;
    jy = 0.0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      r += f[l];
      if (cx_of(l) != 0) jx += cx_of(l) * f[l];
      if (cy_of(l) != 0) jy += cy_of(l) * f[l];
    }
  }
}
#endif

__host__ __device__ inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

}  // namespace lbm

// Kernel launch wrappers (defined in the .cu files, called by lbm_api.cu).
namespace lbm {
struct LaunchCfg {
  int block_warps_y;  // warps per CTA (rows per CTA pass)
  int rows_per_warp;  // rows each warp processes per tile
  int grid_ctas;      // 0: one CTA per tile; else persistent grid size
  int paper_force;    // kernel variant: 0 plain; 1 some member has force kind 2
                      // (BGK collisions); 2 some member has a variable-viscosity
                      // collision (any force); 3 some member has the entropic
                      // collision (with any other collision and force)
  int proj_rows;      // rows per thread of the FP32 four-cell projection (force
                      // kind 2): a block covers 128 x 8 proj_rows cells
};

// One step of every vector-kernel member (flip: tiles in reverse order).
cudaError_t launch_step_f32_vec(const Member *d_members, const Tile *d_tiles, int ntiles,
                                int state, int flip, const LaunchCfg &lc, cudaStream_t s);
cudaError_t launch_step_f32_vec_snap(const Member *d_members, const Tile *d_tiles, int ntiles,
                                     int state, int flip, const LaunchCfg &lc, int slot,
                                     cudaStream_t s);
// rec (optional): the member's public state before the step, FP64
// [9][ny][nx] (the values lbm_get_populations returns), written by the step.
cudaError_t launch_step_scalar(int precision, const Member *d_members, int member,
                               int nx, int ny, int cur, cudaStream_t s, double *rec = nullptr);
struct InitList;
// The general kernel for the members members[0..n) (host array), one launch
// per 256 members, grid sized for nx_max x ny_max.
cudaError_t launch_step_scalar_batch(int precision, const Member *d_members, const int *members,
                                     int n, int nx_max, int ny_max, int state, cudaStream_t s);
// Grid-wide barrier words of the persistent small-grid step (device memory,
// zeroed by each launch): arrival count, generation, error flag.
struct GridSync {
  unsigned *count, *gen;
  int *err;
};
constexpr int kPersistThreads = 32;
constexpr long long kPersistMaxCells = 1LL << 15;  // grids below this take the persistent path
int persistent_ctas(int precision, long long ncells);
cudaError_t barrier_probe(int ctas, int rounds, int withhold, cudaStream_t s, int *gave_up);
cudaError_t launch_step_scalar_persistent(int precision, const Member *d_members, int member,
                                          int state, int nsteps, int ctas, GridSync gs,
                                          cudaStream_t s);
// Member indices of one batched launch (kernel parameter).
struct InitList {
  static constexpr int kMax = 256;
  int n;
  int m[kMax];
};
// Equilibrium initialisation of the n members members[0..n) (host array,
// equal grids nx x ny), member members[i] from rho/ux/uy + i nx ny.
cudaError_t launch_init_fields(int precision, const Member *d_members, const int *members, int n,
                               int nx, int ny, const double *rho, const double *ux,
                               const double *uy, int state, cudaStream_t s);
cudaError_t launch_get_populations(int precision, const Member *d_members, int member,
                                   int nx, int ny, int cur, double *f, cudaStream_t s);
cudaError_t launch_set_populations(int precision, const Member *d_members, int member,
                                   int nx, int ny, int cur, const double *f, cudaStream_t s);
// Damping of eq. (16): the projection of the bare velocity of the current
// state (storage `state`) of every kind-2 member on the 6 mode pairs, then
// the coefficients (kDamp doubles): slot < 0 into Member::damp / damp_f
// (the step about to run), slot 0..2 into that ring slot of damp_ring.
// One launch; members of other kinds are skipped.  quad: the FP32
// four-cell kernel (every kind-2 member with nx % 4 == 0), prow rows per
// thread (>= 1).
cudaError_t launch_projection(int precision, const Member *d_members, int n_members,
                              int nx_max, int ny_max, int state, int slot, bool quad, int prow,
                              cudaStream_t s);
// The ring snapshot of every member in one launch (layout at Member::snap).
cudaError_t launch_snapshot_ring(int precision, const Member *d_members, int n_members,
                                 int nx_max, int ny_max, int state, int slot, bool quad,
                                 cudaStream_t s);
cudaError_t launch_snapshot(int precision, const Member *d_members, int member, int nx,
                            int ny, int cur, double *dst, cudaStream_t s);
cudaError_t launch_status(int precision, const Member *d_members, int member, int nx,
                          int ny, int cur, cudaStream_t s);

// Diagnostics (lbm_diag.cu).  scratch: device FP64 scratch of the handle.
struct DiagScratch {
  double *f;          // slot 0: [nfields][N] field scratch (also general staging)
  size_t N;           // cells of the largest member
  double *partials;   // general reduction partials (kGeneralPartials doubles)
  unsigned *count;    // arrival counter of last-CTA reductions (zero between launches)
  int slots;          // members one batched diagnostic launch covers
  size_t slot_doubles;   // stride of the field slots (slot j at f + j * slot_doubles)
  double *jpart;      // per-slot partials (slot j at jpart + j * jpart_doubles)
  size_t jpart_doubles;
};
constexpr int kDiagFields = 52;
constexpr int kMaxPartialBlocks = 1024;
constexpr int kGeneralPartials = 8 * kMaxPartialBlocks;
constexpr int kDiagMaxL = 32;  // box sizes per balance call
constexpr int kDiagMaxEdges = 256;  // histogram bin edges per quantity

cudaError_t diag_moments(const Member &hm, const double *snap3, double *rho, double *ux,
                         double *uy, double *omega, const DiagScratch &sc, cudaStream_t s);
cudaError_t diag_global(const Member &hm, const double *snap3, const DiagScratch &sc,
                        double *out7_dev, cudaStream_t s);

// One member's share of a batched balance diagnostic.  Every stage runs as
// one launch over all jobs of a batch; the device copy of the job table is
// read by the kernels.
struct DiagJob {
  int nx, ny;
  double nu, alpha, rho_ref;
  const double *fxt, *fyt;     // F_ext,x(y), F_ext,y(x) (FP64 tables)
  const float *fxt_f, *fyt_f;  // the same as FP32 tables (FP32 storage), else NULL
  float nu_f, alpha_f, rho_ref_f;
  const double *s0, *s1, *s2;  // ring snapshots at n, n-1, n-2 (Member::snap
                               // layout; pairs = FP32 (hi, lo) form)
  double *base;                // field slot: term fields and summed-area tables
  double *part;                // partials slot
  const int *meta;             // [nL][8] {L, n_boxes, origin offset (-1: all
                               // periodic origins), per-box row offset,
                               // statistics row, unused x3}
  int nL, max_boxes;
  int force_kind;              // 2: external force = ft64 + damping from dc[level]
  const double *ft64, *trig64; // force kind 2: shell force [2][N], trig tables
  const double *dc[3];         // force kind 2: damping coefficients at n, n-1, n-2
  const float *nu_cell_f;      // variable viscosity: local viscosity at n (FP32
  const double *nu_cell_d;     // or FP64 storage), else both NULL
  int qblocks;                 // query CTAs per (size, balance):
                               // diag_query_blocks(max_boxes, origin list?)
};
// Query CTAs for a job: a fixed function of its own box count, so that the
// statistics do not depend on which members share a batch.
int diag_query_blocks(int max_boxes, bool origin_list, int batch_jobs);
// Doubles of one field slot and of one partials slot for members of at most
// Nmax cells and nx + ny + 1 <= pad.
size_t diag_slot_doubles(size_t Nmax, size_t pad);
size_t diag_job_partials(size_t Nmax, size_t pad);
// The balance diagnostic of G jobs (precision 32: FP32 term arithmetic, 64:
// FP64): term passes, summed-area tables, box queries and statistics, ten
// launches in all.  origins_dev: concatenated (x0, y0) pairs shared by every
// job (NULL when each size uses all periodic origins); stats_dev: rows of
// [15][2] at the statistics rows; per_box_dev only with G == 1.
// Distributions requested from a batched diagnostic: histograms of the
// balancing errors and of the sub-volume Mach number Ma_V (eq. 20), and the
// mean and standard deviation of Ma_V, per statistics row.
struct DiagDist {
  const double *delta_edges, *mach_edges;  // device, ascending, 1..kDiagMaxEdges
  int n_delta, n_mach;
  unsigned long long *hist;  // device [row][3: delta^E, delta^O, Ma_V][kDiagMaxEdges + 1],
                             // zeroed by the caller; counts are added
  double *mach;              // device [row][2]
};
cudaError_t diag_balance(const DiagJob *jobs_host, const DiagJob *jobs_dev, int G,
                         int precision, bool pairs, const int *origins_dev,
                         double *stats_dev, double *per_box_dev, const DiagDist *dist,
                         cudaStream_t s);

// Adjoint (lbm_adjoint.cu).
cudaError_t adjoint_step(const Member &hm, const double *f_n, const double *lam_in,
                         double *lam_out, double w, int bx, int by, int L,
                         double *dJ_dtau, double *dJ_dF0, const DiagScratch &sc,
                         cudaStream_t s);
// The forward objective of the state in storage `state` (acc += w times the
// box average of the dissipation term) in one launch (lbm_adjoint.cu).
cudaError_t objective_tiles(int precision, const Member *d_members, int member,
                            const Member &hm, int state, double w, int bx, int by, int L,
                            double *acc, const DiagScratch &sc, cudaStream_t s);
int adjoint_kernel_count(double w);
// The adjoint steps of a recorded interval, last state first, with one
// gradient reduction per call (weights: host array of nstates).
cudaError_t adjoint_sweep(const Member &hm, const double *states, int nstates,
                          const double *lam_in, double *lam_out, double *lam_tmp,
                          const double *weights, int bx, int by, int L, double *dJ_dtau,
                          double *dJ_dF0, const DiagScratch &sc, cudaStream_t s,
                          long long *launches);
cudaError_t probe_fma_rate(int bits, cudaStream_t s, double *flops_per_s);
}  // namespace lbm
