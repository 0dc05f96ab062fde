// Sub-volume energy/enstrophy balance diagnostic of Tauzin et al. (2018):
// the local terms of eqs. (8)-(11) in 2D with the eq. (18) 8th-order
// centred differences and the eq. (17) BDF2 time derivative, their L x L box
// averages through FP64 summed-area tables (O(1) per box and size), the
// balancing errors of eqs. (12), (13) and their statistics per box size.
//
// Inputs are moment snapshots (rho, j_x, j_y) in FP64, layout [3][ny*nx].
// All diagnostic arithmetic is FP64.  Scratch layout: fields of N = nx*ny
// doubles at sc.f + k*N (k < kDiagFields), reduction partials at
// sc.partials.
#include <cmath>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

enum Field {
  S_RHO = 0, S_JX, S_JY,      // temporary snapshot (moments / global)
  U0X, U0Y, U1X, U1Y, U2X, U2Y,
  R0, FXR, FYR, PP, A1, A2, WW, B1, B2, C1, C2, G1, G2, G3, K1, K2,
  T0,                         // T0..T11: term fields 0..11 (term 12 is 0)
  NFIELDS = T0 + 12
};
static_assert(NFIELDS <= kDiagFields, "scratch too small");

struct Grid {
  int nx, ny;
  double nu, alpha;
  const double *fxt, *fyt;  // F_ext,x(y), F_ext,y(x)
};

__device__ __forceinline__ int wrapn(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Eq. (18) in x and y (dx = 1), periodic; paired form of the same stencil:
// 4/5 (A+1 - A-1) - 1/5 (A+2 - A-2) + 4/105 (A+3 - A-3) - 1/280 (A+4 - A-4).
__device__ __forceinline__ double ddx(const double *A, const Grid &g, int x, int y) {
  const double *r = A + (size_t)y * g.nx;
  double a[9];
#pragma unroll
  for (int d = -4; d <= 4; ++d) a[d + 4] = r[g.nx >= 4 ? wrapn(x + d, g.nx) : wrapi(x + d, g.nx)];
  return 0.8 * (a[5] - a[3]) - 0.2 * (a[6] - a[2]) + (4.0 / 105.0) * (a[7] - a[1]) -
         (1.0 / 280.0) * (a[8] - a[0]);
}
__device__ __forceinline__ double ddy(const double *A, const Grid &g, int x, int y) {
  double a[9];
#pragma unroll
  for (int d = -4; d <= 4; ++d)
    a[d + 4] = A[(size_t)(g.ny >= 4 ? wrapn(y + d, g.ny) : wrapi(y + d, g.ny)) * g.nx + x];
  return 0.8 * (a[5] - a[3]) - 0.2 * (a[6] - a[2]) + (4.0 / 105.0) * (a[7] - a[1]) -
         (1.0 / 280.0) * (a[8] - a[0]);
}

__device__ __forceinline__ double bdf2(double a0, double a1, double a2) {
  return (3.0 * a0 - 4.0 * a1 + a2) * 0.5;  // eq. (17), dt = 1
}

#define CELL_INDEX                                        \
  const int x = blockIdx.x * blockDim.x + threadIdx.x;    \
  const int y = blockIdx.y * blockDim.y + threadIdx.y;    \
  if (x >= g.nx || y >= g.ny) return;                     \
  const size_t c = (size_t)y * g.nx + x;

// Velocity u = (j + F/2)/rho with F = F_ext - alpha j.
__device__ __forceinline__ void phys_velocity(const Grid &g, int x, int y, double r, double jx,
                                              double jy, double &ux, double &uy, double &Fx,
                                              double &Fy) {
  Fx = g.fxt[y] - g.alpha * jx;
  Fy = g.fyt[x] - g.alpha * jy;
  ux = (jx + 0.5 * Fx) / r;
  uy = (jy + 0.5 * Fy) / r;
}

// Pass 0 (pointwise): velocities at n, n-1, n-2; LHS^E, RHS^{E,3}; fluxes
// of E; F / rho; p.
__global__ void k_prep(Grid g, const double *s0, const double *s1, const double *s2,
                       double *F, size_t N) {
  CELL_INDEX;
  const double *sn[3] = {s0, s1, s2};
  double E[3], u0 = 0, v0 = 0, Fx0 = 0, Fy0 = 0;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double r = sn[m][c], jx = sn[m][N + c], jy = sn[m][2 * N + c];
    double u, v, Fx, Fy;
    phys_velocity(g, x, y, r, jx, jy, u, v, Fx, Fy);
    F[(U0X + 2 * m) * N + c] = u;
    F[(U0Y + 2 * m) * N + c] = v;
    E[m] = 0.5 * r * (u * u + v * v);
    if (m == 0) { u0 = u; v0 = v; Fx0 = Fx; Fy0 = Fy; }
  }
  const double r = s0[c];
  F[R0 * N + c] = r;
  F[FXR * N + c] = Fx0 / r;
  F[FYR * N + c] = Fy0 / r;
  F[PP * N + c] = r / 3.0;  // p = cs^2 rho
  F[A1 * N + c] = E[0] * u0;
  F[A2 * N + c] = E[0] * v0;
  F[(T0 + 0) * N + c] = bdf2(E[0], E[1], E[2]);  // LHS^E
  F[(T0 + 3) * N + c] = u0 * Fx0 + v0 * Fy0;     // RHS^{E,3} = u.F
}

// Pass 1 (radius 4): vorticity at three levels, LHS^Omega, velocity
// gradients, RHS^{E,2}, RHS^{E,4}, RHS^{O,2}, RHS^{O,3}; fluxes for pass 2.
__global__ void k_grad(Grid g, double *F, size_t N) {
  CELL_INDEX;
  double w[3];
#pragma unroll
  for (int m = 0; m < 3; ++m)
    w[m] = ddx(F + (U0Y + 2 * m) * N, g, x, y) - ddy(F + (U0X + 2 * m) * N, g, x, y);
  const double Om = 0.5 * w[0] * w[0];
  F[(T0 + 6) * N + c] = bdf2(Om, 0.5 * w[1] * w[1], 0.5 * w[2] * w[2]);  // LHS^O
  const double *U = F + U0X * N, *V = F + U0Y * N;
  const double dxu = ddx(U, g, x, y), dyu = ddy(U, g, x, y);
  const double dxv = ddx(V, g, x, y), dyv = ddy(V, g, x, y);
  const double u = U[c], v = V[c], r = F[R0 * N + c];
  const double sxx = 2.0 * dxu, sxy = dyu + dxv, syy = 2.0 * dyv;  // S_ij = d_j u_i + d_i u_j
  const double nr = g.nu * r;
  F[(T0 + 2) * N + c] = -(u * ddx(F + PP * N, g, x, y) + v * ddy(F + PP * N, g, x, y));
  F[(T0 + 4) * N + c] = -nr * (sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv);
  F[(T0 + 8) * N + c] = -Om * (dxu + dyv);
  F[(T0 + 9) * N + c] = w[0] * (ddx(F + FYR * N, g, x, y) - ddy(F + FXR * N, g, x, y));
  F[WW * N + c] = w[0];
  F[B1 * N + c] = Om * u;
  F[B2 * N + c] = Om * v;
  F[C1 * N + c] = nr * (u * sxx + v * sxy);
  F[C2 * N + c] = nr * (u * sxy + v * syy);
  F[G1 * N + c] = nr * sxx;
  F[G2 * N + c] = nr * sxy;
  F[G3 * N + c] = nr * syy;
}

// Pass 2 (radius 4): flux divergences RHS^{E,1}, RHS^{E,5}, RHS^{O,1}; H_i;
// RHS^{O,4}; products w H for pass 3.
__global__ void k_flux(Grid g, double *F, size_t N) {
  CELL_INDEX;
  const double r = F[R0 * N + c];
  F[(T0 + 1) * N + c] = -(ddx(F + A1 * N, g, x, y) + ddy(F + A2 * N, g, x, y));
  F[(T0 + 5) * N + c] = ddx(F + C1 * N, g, x, y) + ddy(F + C2 * N, g, x, y);
  F[(T0 + 7) * N + c] = -(ddx(F + B1 * N, g, x, y) + ddy(F + B2 * N, g, x, y));
  const double Hx = (ddx(F + G1 * N, g, x, y) + ddy(F + G2 * N, g, x, y)) / r;
  const double Hy = (ddx(F + G2 * N, g, x, y) + ddy(F + G3 * N, g, x, y)) / r;
  const double *W = F + WW * N;
  F[(T0 + 10) * N + c] = Hx * ddy(W, g, x, y) - Hy * ddx(W, g, x, y);
  const double w = W[c];
  F[K1 * N + c] = w * Hy;
  F[K2 * N + c] = w * Hx;
}

// Pass 3 (radius 4): RHS^{O,5} = d_x (w H_y) - d_y (w H_x).
__global__ void k_curl(Grid g, double *F, size_t N) {
  CELL_INDEX;
  F[(T0 + 11) * N + c] = ddx(F + K1 * N, g, x, y) - ddy(F + K2 * N, g, x, y);
}

// ---------------------------------------------------------------------------
// Moments and whole-grid quantities
// ---------------------------------------------------------------------------

__global__ void k_moments(Grid g, const double *snap, size_t N, double *rho, double *ux,
                          double *uy) {
  CELL_INDEX;
  const double r = snap[c];
  double u, v, Fx, Fy;
  phys_velocity(g, x, y, r, snap[N + c], snap[2 * N + c], u, v, Fx, Fy);
  if (rho) rho[c] = r;
  ux[c] = u;
  uy[c] = v;
}

__global__ void k_vorticity(Grid g, const double *ux, const double *uy, double *omega) {
  CELL_INDEX;
  omega[c] = ddx(uy, g, x, y) - ddy(ux, g, x, y);
}

// Block-deterministic sums: each block writes its partial for every
// quantity; a single-block pass adds the partials in index order.
template <int NQ>
__device__ void block_sum_store(double (&v)[NQ], double *out /*[NQ]*/) {
  __shared__ double sh[NQ][32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double a = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = a;
  }
  __syncthreads();
  if (tid < NQ) {
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a += sh[tid][k];
    out[tid] = a;
  }
}

__global__ void k_global(Grid g, const double *snap, const double *ux, const double *uy,
                         size_t N, double *partials) {
  // grid-stride over cells, fixed order per block
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  for (size_t c = (size_t)blockIdx.x * nthr + tid; c < N; c += (size_t)gridDim.x * nthr) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    const double r = snap[c], jx = snap[N + c], jy = snap[2 * N + c];
    const double Fx = g.fxt[y] - g.alpha * jx, Fy = g.fyt[x] - g.alpha * jy;
    const double u = ux[c], v = uy[c];
    const double dxu = ddx(ux, g, x, y), dyu = ddy(ux, g, x, y);
    const double dxv = ddx(uy, g, x, y), dyv = ddy(uy, g, x, y);
    const double w = dxv - dyu;
    const double sxx = 2 * dxu, sxy = dyu + dxv, syy = 2 * dyv;
    acc[0] += r;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += 0.5 * r * (u * u + v * v);
    acc[4] += 0.5 * w * w;
    acc[5] += u * Fx + v * Fy;
    acc[6] += g.nu * r * (sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv);
  }
  block_sum_store<7>(acc, partials + (size_t)blockIdx.x * 7);
}

__global__ void k_global_final(const double *partials, int nblocks, size_t N, double *out) {
  const int q = threadIdx.x;
  if (q >= 7) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) a += partials[(size_t)b * 7 + q];
  out[q] = q < 3 ? a : a / (double)N;
}

// ---------------------------------------------------------------------------
// Summed-area tables
// ---------------------------------------------------------------------------

// Per-field sums (for the mean subtracted before the scan).
__global__ void k_field_sums(const double *T, size_t N, double *partials) {
  const int f = blockIdx.y;
  const double *A = T + (size_t)f * N;
  double a[1] = {0.0};
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    a[0] += A[i];
  block_sum_store<1>(a, partials + (size_t)f * gridDim.x + blockIdx.x);
}

__global__ void k_field_means(const double *partials, int nblocks, size_t N, double *means,
                              int nf) {
  const int f = threadIdx.x;
  if (f >= nf) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) a += partials[(size_t)f * nblocks + b];
  means[f] = a / (double)N;
}

// Inclusive scan along x of (T - mean), one CTA (256 threads) per (row, field).
__global__ void __launch_bounds__(256) k_sat_rows(double *T, int nx, int ny,
                                                  const double *means) {
  const int y = blockIdx.x, f = blockIdx.y;
  double *row = T + ((size_t)f * ny + y) * nx;
  const double mean = means[f];
  __shared__ double wsum[8];
  __shared__ double carry_sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double carry = 0.0;
  for (int base = 0; base < nx; base += 256) {
    const int x = base + tid;
    double v = x < nx ? row[x] - mean : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double n = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += n;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    double off = carry;
    for (int k = 0; k < wid; ++k) off += wsum[k];
    if (x < nx) row[x] = v + off;
    if (tid == 255) {
      double tot = carry;
      for (int k = 0; k < 8; ++k) tot += wsum[k];
      carry_sh = tot;
    }
    __syncthreads();
    carry = carry_sh;
    __syncthreads();
  }
}

// Inclusive scan along y over a strip of 32 columns of one field: the 8
// warps of the CTA each sum one chunk of rows, exchange the chunk totals
// through shared memory, then rewrite their chunk as a running sum started
// from the total of the chunks above.  Loads are coalesced across the strip.
__global__ void __launch_bounds__(256) k_sat_cols(double *T, int nx, int ny) {
  const int f = blockIdx.y;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int w = threadIdx.y;
  const int chunk = (ny + 7) / 8;
  const int y0 = min(ny, w * chunk), y1 = min(ny, y0 + chunk);
  double *col = T + (size_t)f * nx * ny + x;
  __shared__ double tot[8][32];
  double s = 0.0;
  if (x < nx) {
    int y = y0;
    for (; y + 8 <= y1; y += 8) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = col[(size_t)(y + k) * nx];
#pragma unroll
      for (int k = 0; k < 8; ++k) s += v[k];
    }
    for (; y < y1; ++y) s += col[(size_t)y * nx];
  }
  tot[w][threadIdx.x] = s;
  __syncthreads();
  double acc = 0.0;
  for (int k = 0; k < w; ++k) acc += tot[k][threadIdx.x];
  if (x < nx) {
    int y = y0;
    for (; y + 8 <= y1; y += 8) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = col[(size_t)(y + k) * nx];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        acc += v[k];
        col[(size_t)(y + k) * nx] = acc;
      }
    }
    for (; y < y1; ++y) {
      acc += col[(size_t)y * nx];
      col[(size_t)y * nx] = acc;
    }
  }
}

// Exclusive prefix P(x, y) = sum over x' < x, y' < y, from the inclusive
// table S, for 0 <= x <= nx, 0 <= y <= ny.
__device__ __forceinline__ double Pex(const double *S, int nx, int x, int y) {
  return (x == 0 || y == 0) ? 0.0 : S[(size_t)(y - 1) * nx + (x - 1)];
}
// Prefix over the periodic extension, 0 <= x < 2 nx, 0 <= y < 2 ny.
__device__ __forceinline__ double Pext(const double *S, int nx, int ny, int x, int y) {
  const int qx = x >= nx, qy = y >= ny;
  const int xm = x - qx * nx, ym = y - qy * ny;
  double v = Pex(S, nx, xm, ym);
  if (qx) v += Pex(S, nx, nx, ym);
  if (qy) v += Pex(S, nx, xm, ny);
  if (qx && qy) v += Pex(S, nx, nx, ny);
  return v;
}

// Balancing error of eqs. (12), (13) from the box LHS, the running sum of
// the RHS terms and their largest magnitude.
__device__ __forceinline__ double delta_of(double lhs, double sum, double mx) {
  const double num = fabs(sum - lhs);
  if (mx == 0.0) return num == 0.0 ? 0.0 : INFINITY;
  return num / mx;
}

constexpr int kQStats = 28;  // [dE, dE^2, dZ, dZ^2, (d_k, d_k^2) for the 12 fields]

// One thread per box: the 12 non-zero box averages (term 12, the 2D
// vortex-stretching term, is identically 0), the two balancing errors, sums
// of the deviations from the field means and of their squares for the
// statistics, and optionally the per-box values.
template <bool PER_BOX>
__global__ void __launch_bounds__(256) k_query(const double *__restrict__ T, int nx, int ny,
                                               const double *__restrict__ means,
                                               const int *__restrict__ Ls, int nb,
                                               const int *__restrict__ origins,
                                               double *partials, double *per_box) {
  const int iL = blockIdx.y;
  const int L = Ls[iL];
  const size_t N = (size_t)nx * ny;
  const double invA = 1.0 / ((double)L * (double)L);
  double mean[12], s1[12], s2[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    mean[k] = means[k];
    s1[k] = 0.0;
    s2[k] = 0.0;
  }
  double dE1 = 0.0, dE2 = 0.0, dZ1 = 0.0, dZ2 = 0.0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const int x0 = origins ? origins[2 * b] : b % nx;
    const int y0 = origins ? origins[2 * b + 1] : b / nx;
    double lhsE = 0.0, sumE = 0.0, maxE = 0.0, lhsZ = 0.0, sumZ = 0.0, maxZ = 0.0;
    double *o = PER_BOX ? per_box + ((size_t)iL * nb + b) * 15 : nullptr;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const double *S = T + (size_t)k * N;
      const double d = (Pext(S, nx, ny, x0 + L, y0 + L) - Pext(S, nx, ny, x0, y0 + L) -
                        Pext(S, nx, ny, x0 + L, y0) + Pext(S, nx, ny, x0, y0)) * invA;
      const double v = d + mean[k];
      s1[k] += d;
      s2[k] += d * d;
      if (k == 0) {
        lhsE = v;
      } else if (k < 6) {
        sumE += v;
        maxE = fmax(maxE, fabs(v));
      } else if (k == 6) {
        lhsZ = v;
      } else {
        sumZ += v;
        maxZ = fmax(maxZ, fabs(v));
      }
      if (PER_BOX) o[2 + k] = v;
    }
    const double dE = delta_of(lhsE, sumE, maxE), dZ = delta_of(lhsZ, sumZ, maxZ);
    dE1 += dE;
    dE2 += dE * dE;
    dZ1 += dZ;
    dZ2 += dZ * dZ;
    if (PER_BOX) {
      o[0] = dE;
      o[1] = dZ;
      o[14] = 0.0;
    }
  }
  double acc[kQStats];
  acc[0] = dE1;
  acc[1] = dE2;
  acc[2] = dZ1;
  acc[3] = dZ2;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    acc[4 + 2 * k] = s1[k];
    acc[5 + 2 * k] = s2[k];
  }
  block_sum_store<kQStats>(acc, partials + ((size_t)iL * gridDim.x + blockIdx.x) * kQStats);
}

// Mean and population standard deviation of the 15 quantities per size.
__global__ void k_stats_final(const double *partials, int nblocks, const double *means,
                              int nb, int nL, double *stats) {
  const int iL = blockIdx.x, q = threadIdx.x;
  if (q >= 15) return;
  double mean = 0.0, sd = 0.0;
  if (q < 14) {
    const int i = q < 2 ? 2 * q : 4 + 2 * (q - 2);
    double s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      s1 += partials[((size_t)iL * nblocks + b) * kQStats + i];
      s2 += partials[((size_t)iL * nblocks + b) * kQStats + i + 1];
    }
    const double m1 = s1 / nb;
    const double shift = q >= 2 ? means[q - 2] : 0.0;
    mean = shift + m1;
    sd = sqrt(fmax(s2 / nb - m1 * m1, 0.0));
  }
  stats[((size_t)iL * 15 + q) * 2] = mean;
  stats[((size_t)iL * 15 + q) * 2 + 1] = sd;
}

Grid grid_of(const Member &hm) {
  Grid g;
  g.nx = hm.nx;
  g.ny = hm.ny;
  g.nu = hm.nu;
  g.alpha = hm.alpha;
  g.fxt = hm.fx_tab64;
  g.fyt = hm.fy_tab64;
  return g;
}

dim3 cells_grid(const Grid &g, dim3 b) {
  return dim3((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y);
}

}  // namespace

cudaError_t diag_moments(const Member &hm, const double *snap3, double *rho, double *ux,
                         double *uy, double *omega, const DiagScratch &sc, cudaStream_t s) {
  const Grid g = grid_of(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  double *U = ux ? ux : sc.f + (size_t)U0X * N;
  double *V = uy ? uy : sc.f + (size_t)U0Y * N;
  dim3 b(32, 8);
  k_moments<<<cells_grid(g, b), b, 0, s>>>(g, snap3, N, rho, U, V);
  if (omega) k_vorticity<<<cells_grid(g, b), b, 0, s>>>(g, U, V, omega);
  return cudaGetLastError();
}

cudaError_t diag_global(const Member &hm, const double *snap3, const DiagScratch &sc,
                        double *out7_dev, cudaStream_t s) {
  const Grid g = grid_of(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  double *U = sc.f + (size_t)U0X * N, *V = sc.f + (size_t)U0Y * N;
  dim3 b(32, 8);
  k_moments<<<cells_grid(g, b), b, 0, s>>>(g, snap3, N, nullptr, U, V);
  int nblocks = (int)((N + 255) / 256);
  if (nblocks > kMaxPartialBlocks) nblocks = kMaxPartialBlocks;
  k_global<<<nblocks, dim3(32, 8), 0, s>>>(g, snap3, U, V, N, sc.partials);
  k_global_final<<<1, 32, 0, s>>>(sc.partials, nblocks, N, out7_dev);
  return cudaGetLastError();
}

cudaError_t diag_terms(const Member &hm, const double *sn, const double *sn1,
                       const double *sn2, const DiagScratch &sc, cudaStream_t s) {
  const Grid g = grid_of(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  dim3 b(32, 8), gr = cells_grid(g, b);
  k_prep<<<gr, b, 0, s>>>(g, sn, sn1, sn2, sc.f, N);
  k_grad<<<gr, b, 0, s>>>(g, sc.f, N);
  k_flux<<<gr, b, 0, s>>>(g, sc.f, N);
  k_curl<<<gr, b, 0, s>>>(g, sc.f, N);
  return cudaGetLastError();
}

double *diag_term_fields(const DiagScratch &sc, size_t N) { return sc.f + (size_t)T0 * N; }

size_t diag_partials_needed(int nL) {
  return (size_t)12 * kMaxPartialBlocks + 16 + (size_t)nL * kMaxPartialBlocks * 30 +
         (size_t)nL * 30;
}

// SAT of the 12 term fields (in place) and the box queries for every L.
// Ls_dev and origins_dev are device arrays; stats_dev receives [nL][15][2].
cudaError_t diag_sat_and_query(const Member &hm, const int *Ls_dev, int nL,
                               const int *origins_dev, int n_origins,
                               const DiagScratch &sc, double *stats_dev,
                               double *per_box_dev, cudaStream_t s) {
  const int nx = hm.nx, ny = hm.ny;
  const size_t N = (size_t)nx * ny;
  double *T = sc.f + (size_t)T0 * N;
  double *part_means = sc.partials;                       // [12][kMaxPartialBlocks]
  double *means = part_means + 12 * kMaxPartialBlocks;    // [12] (+4 pad)
  double *part_q = means + 16;                            // [nL][blocks][30]
  // about 16 elements per thread for the field sums
  int nb_sum = (int)((N + 4095) / 4096);
  if (nb_sum > kMaxPartialBlocks) nb_sum = kMaxPartialBlocks;
  k_field_sums<<<dim3(nb_sum, 12), 256, 0, s>>>(T, N, part_means);
  k_field_means<<<1, 32, 0, s>>>(part_means, nb_sum, N, means, 12);
  k_sat_rows<<<dim3(ny, 12), 256, 0, s>>>(T, nx, ny, means);
  k_sat_cols<<<dim3((nx + 31) / 32, 12), dim3(32, 8), 0, s>>>(T, nx, ny);
  const int nbox = origins_dev ? n_origins : (int)N;
  // about 4 boxes per thread, at most kMaxPartialBlocks CTAs per size
  int qblocks = (nbox + 1023) / 1024;
  if (qblocks > kMaxPartialBlocks) qblocks = kMaxPartialBlocks;
  if (qblocks < 1) qblocks = 1;
  if (per_box_dev)
    k_query<true><<<dim3(qblocks, nL), 256, 0, s>>>(T, nx, ny, means, Ls_dev, nbox,
                                                    origins_dev, part_q, per_box_dev);
  else
    k_query<false><<<dim3(qblocks, nL), 256, 0, s>>>(T, nx, ny, means, Ls_dev, nbox,
                                                     origins_dev, part_q, nullptr);
  k_stats_final<<<nL, 32, 0, s>>>(part_q, qblocks, means, nbox, nL, stats_dev);
  return cudaGetLastError();
}

}  // namespace lbm
