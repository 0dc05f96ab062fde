// Reverse mode of the D2Q9 BGK + exact-difference-forcing step (eq. (1),
// eq. (2), Sec. 3 of Tauzin et al. 2018) and of the box-averaged
// dissipation objective built from the RHS^{E,4} term of eq. (8).  This is
// the differentiation of the forward model; the paper has no counterpart.
//
// Forward step in the public layout (f = pre-collision state):
//   f*_l(x) = (1 - w) f_l + (w - 1) feq_l(rho, j) + feq_l(rho, m'),
//   f_l(x + c_l, n+1) = f*_l(x),
// with w = 1/tau, rho = sum f, j = sum c f, m' = (1 - alpha) j + F_ext
// (= rho (u + F/rho)), and the equilibrium written in momentum form
//   feq_l(rho, m) = t_l [rho + 3 c.m + (4.5 (c.m)^2 - 1.5 |m|^2) / rho].
// Adjoint: mu_l(x) = lambda_l(x + c_l, n+1) (transpose of the push), then
//   lambda_l(x, n) = (1 - w) mu_l + A_rho + c_l . A_j + dJ_n/df_l(x),
//   A_rho = sum_k mu_k [(w - 1) d_rho feq_k(rho, j) + d_rho feq_k(rho, m')],
//   A_j   = sum_k mu_k [(w - 1) d_m feq_k(rho, j) + (1 - alpha) d_m feq_k(rho, m')],
//   dJ/dtau += sum mu_l (f_l - feq_l(rho, j)) / tau^2,
//   dJ/dF0  += sum mu_l d_m feq_l(rho, m') . s,  s = (sin(2 pi kf y/ny), sin(2 pi kf x/nx)).
// Objective term at time n: J_n = weight / L^2 * sum_{x in box} eps(x),
//   eps = -nu rho S_ij G_ij, G_ij = D_j u_i, S_ij = G_ij + G_ji,
//   u = (j + F/2)/rho, F = F_ext - alpha j, nu = (tau - 1/2)/3,
// whose adjoint uses D^T = -D (antisymmetric periodic eq. (18) stencil).
// All arithmetic is FP64; reductions are block-deterministic.
#include <algorithm>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

enum AdjField { A_RHO = 0, A_JX, A_JY, A_U, A_V, GAM_XX, GAM_XY, GAM_YY, D_RHO, D_JX, D_JY,
                D_TOT, S_TAB, A_NFIELDS };  // S_TAB: sin(2 pi kf y/ny) [ny], then of x [nx]
static_assert(A_NFIELDS <= kDiagFields, "scratch too small");

struct AGrid {
  int nx, ny, kf, force;
  double nu, alpha, tau, omega, F0;
  const double *fxt, *fyt;  // F_ext tables (F0 included)
};

__device__ __forceinline__ int wrapn(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}
__device__ __forceinline__ int wr(int i, int n) { return n >= 4 ? wrapn(i, n) : wrapi(i, n); }

__device__ __forceinline__ void force_dir(const AGrid &g, int x, int y, double &sx, double &sy) {
  if (g.force == 1) {
    sx = sinpi(2.0 * g.kf * (double)y / g.ny);
    sy = sinpi(2.0 * g.kf * (double)x / g.nx);
  } else {
    sx = 0.0;
    sy = 0.0;
  }
}

// The direction s of dF_ext/dF0 per row and column, tabulated once per
// adjoint step (the cell kernel then reads two doubles instead of
// evaluating two FP64 sines, which the FP64 pipe of this part pays for).
__global__ void k_sine_tables(AGrid g, double *tab) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.ny + g.nx;
       i += gridDim.x * blockDim.x) {
    double sx, sy;
    if (i < g.ny) {
      force_dir(g, 0, i, sx, sy);
      tab[i] = sx;
    } else {
      force_dir(g, i - g.ny, 0, sx, sy);
      tab[i] = sy;
    }
  }
}

template <int NQ>
__device__ void block_sums(double (&v)[NQ], double *out, int add = 0) {
  __shared__ double sh[NQ][32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
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
    out[tid] = add ? out[tid] + a : a;
  }
}

#define FOR_CELLS                                                                   \
  const size_t N = (size_t)g.nx * g.ny;                                             \
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;             \
       c += (size_t)gridDim.x * blockDim.x)

// The objective touches only the box V0 and the cells within the eq. (18)
// stencil reach (4 cells) of it: the region R = V0 widened by 4 on each
// side (the whole axis where that covers it).  u is needed on R, Gamma on
// V0 and dJ/du = -D^T Gamma on R; every other cell has no objective term.
struct Region {
  int x0, y0, w, h;  // lower-left corner (wrapped) and extent, w <= nx, h <= ny
};

__host__ __device__ inline Region objective_region(int nx, int ny, int bx, int by, int L) {
  Region r;
  if (L + 8 >= nx) { r.x0 = 0; r.w = nx; } else { r.x0 = ((bx - 4) % nx + nx) % nx; r.w = L + 8; }
  if (L + 8 >= ny) { r.y0 = 0; r.h = ny; } else { r.y0 = ((by - 4) % ny + ny) % ny; r.h = L + 8; }
  return r;
}

__device__ __forceinline__ bool in_region(int x, int y, const Region &r, const AGrid &g) {
  return wrapi(x - r.x0, g.nx) < r.w && wrapi(y - r.y0, g.ny) < r.h;
}

#define FOR_REGION(R)                                                                  \
  const size_t N = (size_t)g.nx * g.ny;                                                \
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (R).w * (R).h;               \
       i += gridDim.x * blockDim.x)

// rho, j and u = (j + F/2)/rho of the public state f[9][ny][nx] on R.
__global__ void k_region_velocity(AGrid g, Region R, const double *f, double *F) {
  FOR_REGION(R) {
    const int x = wrapi(R.x0 + i % R.w, g.nx), y = wrapi(R.y0 + i / R.w, g.ny);
    const size_t c = (size_t)y * g.nx + x;
    double r = 0, a = 0, b = 0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const double v = f[(size_t)l * N + c];
      r += v;
      if (cx_of(l) != 0) a += cx_of(l) * v;
      if (cy_of(l) != 0) b += cy_of(l) * v;
    }
    const double Fx = g.fxt[y] - g.alpha * a, Fy = g.fyt[x] - g.alpha * b;
    const double ir = 1.0 / r;
    F[A_RHO * N + c] = r;
    F[A_U * N + c] = (a + 0.5 * Fx) * ir;
    F[A_V * N + c] = (b + 0.5 * Fy) * ir;
  }
}

// Four lanes per cell: lanes 4q .. 4q + 3 of a warp share cell q of the
// warp's group of eight, lane part p = lane & 3 evaluates one of the cell's
// four stencil derivatives and the quad exchanges them by shuffles (a
// quarter of the dependent FP64 chain per lane, four times the SMs).  The
// loop runs in whole warps: a lane past the last cell works on the last
// cell and writes nothing, so every shuffle has the full warp.
#define FOR_QUADS(NCELLS)                                                      \
  const int lane = threadIdx.x & 31, p = lane & 3, qb = lane & ~3;             \
  const int wglob = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);       \
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);                     \
  for (int i0 = wglob * 8; i0 < (NCELLS); i0 += nwarps * 8)

__device__ __forceinline__ double quad_get(double v, int qb, int k) {
  return __shfl_sync(0xffffffffu, v, qb + k);
}

// The eq. (18) stencil derivative of A along x (dir 0) or y (dir 1) at (x, y),
// one code path for both directions (no divergence within a quad).
__device__ __forceinline__ double D_dir(const double *A, const AGrid &g, int x, int y, int dir) {
  auto at = [&](int k) {
    return dir ? A[(size_t)wr(y + k, g.ny) * g.nx + x] : A[(size_t)y * g.nx + wr(x + k, g.nx)];
  };
  return 0.8 * (at(1) - at(-1)) - 0.2 * (at(2) - at(-2)) + (4.0 / 105.0) * (at(3) - at(-3)) -
         (1.0 / 280.0) * (at(4) - at(-4));
}

// Objective pass 1, over V0: Gamma_ij = dJ/dG_ij = -2 c nu rho S_ij
// (c = weight / L^2); explicit dJ/dtau part -c rho Q / 3 (d nu / d tau = 1/3).
// Four lanes per cell (FOR_QUADS): d/dx u, d/dy u, d/dx v, d/dy v.
__global__ void k_obj_gamma(AGrid g, double *F, double cw, int bx, int by, int L,
                            double *partials, int add) {
  double acc[1] = {0.0};
  const size_t N = (size_t)g.nx * g.ny;
  const int nc = L * L;
  FOR_QUADS(nc) {
    const int iq = i0 + (lane >> 2), i = iq < nc ? iq : nc - 1;
    const int x = wrapi(bx + i % L, g.nx), y = wrapi(by + i / L, g.ny);
    const size_t c = (size_t)y * g.nx + x;
    const double d = D_dir(F + (p < 2 ? A_U : A_V) * N, g, x, y, p & 1);
    const double dxu = quad_get(d, qb, 0), dyu = quad_get(d, qb, 1);
    const double dxv = quad_get(d, qb, 2), dyv = quad_get(d, qb, 3);
    if (iq < nc) {
      const double sxx = 2 * dxu, sxy = dyu + dxv, syy = 2 * dyv;
      const double r = F[A_RHO * N + c];
      if (p < 3) {  // Gamma_xx, Gamma_xy, Gamma_yy: one per lane
        const double sp = p == 0 ? sxx : (p == 1 ? sxy : syy);
        F[(GAM_XX + p) * N + c] = -2.0 * cw * g.nu * r * sp;
      } else {
        const double Q = sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv;
        F[D_RHO * N + c] = -cw * g.nu * Q;
        acc[0] += -cw * r * Q / 3.0;
      }
    }
  }
  block_sums<1>(acc, partials + blockIdx.x, add);
}

// Objective pass 2, over R: dJ/du_i = -sum_j D_j Gamma_ij (D^T = -D), then
// dJ/drho (with the direct part of V0), dJ/dj and the explicit dJ/dF0 part
// through u = ((1 - alpha/2) j + F_ext/2)/rho.  Four lanes per cell
// (FOR_QUADS): D_x Gamma_xx, D_y Gamma_xy, D_x Gamma_xy, D_y Gamma_yy, Gamma
// zero outside V0; then one quotient per lane (dJ/djx, dJ/djy, the velocity
// part of dJ/drho, the dJ/dF0 term) and the force direction s from the
// sine tables at F[S_TAB].
__global__ void k_obj_velocity_adjoint(AGrid g, Region R, double *F, int bx, int by, int L,
                                       double *partials, int add) {
  double acc[1] = {0.0};
  const size_t N = (size_t)g.nx * g.ny;
  const int nc = R.w * R.h;
  FOR_QUADS(nc) {
    const int iq = i0 + (lane >> 2), i = iq < nc ? iq : nc - 1;
    const int x = wrapi(R.x0 + i % R.w, g.nx), y = wrapi(R.y0 + i / R.w, g.ny);
    const size_t c = (size_t)y * g.nx + x;
    // box-relative coordinates: the stencil point k along dir is in V0 when
    // its along coordinate wraps into [0, L) and the cross one already is
    const int rx = wrapi(x - bx, g.nx), ry = wrapi(y - by, g.ny);
    const int dir = p & 1;
    const double *G = F + (p == 0 ? GAM_XX : (p == 3 ? GAM_YY : GAM_XY)) * N;
    const int ra = dir ? ry : rx, na = dir ? g.ny : g.nx;
    const bool cross_in = (dir ? rx : ry) < L;
    auto at = [&](int k) {
      const int t = wr(ra + k, na);
      const size_t e = dir ? (size_t)wr(y + k, g.ny) * g.nx + x : (size_t)y * g.nx + wr(x + k, g.nx);
      return (cross_in && t < L) ? G[e] : 0.0;
    };
    const double d = 0.8 * (at(1) - at(-1)) - 0.2 * (at(2) - at(-2)) +
                     (4.0 / 105.0) * (at(3) - at(-3)) - (1.0 / 280.0) * (at(4) - at(-4));
    const double Ux = -(quad_get(d, qb, 0) + quad_get(d, qb, 1));
    const double Uy = -(quad_get(d, qb, 2) + quad_get(d, qb, 3));
    const double r = F[A_RHO * N + c];
    double num;
    if (p == 0) {
      num = Ux * (1.0 - 0.5 * g.alpha);
    } else if (p == 1) {
      num = Uy * (1.0 - 0.5 * g.alpha);
    } else if (p == 2) {
      num = Ux * F[A_U * N + c] + Uy * F[A_V * N + c];
    } else {
      num = Ux * F[S_TAB * N + y] + Uy * F[S_TAB * N + g.ny + x];
    }
    const double q = num / (p == 3 ? 2.0 * r : r);
    if (iq < nc) {
      if (p < 2) {
        F[(D_JX + p) * N + c] = q;
      } else if (p == 2) {
        const double direct = (rx < L && ry < L) ? F[D_RHO * N + c] : 0.0;
        F[D_TOT * N + c] = direct - q;
      } else {
        acc[0] += q;
      }
    }
  }
  block_sums<1>(acc, partials + blockIdx.x, add);
}

// t_l-weighted sums over the populations of the pulled adjoint mu_l and
// their contractions with the equilibrium's derivatives.  With
//   feq_l(rho, m) = t_l [rho + 3 c.m + (4.5 (c.m)^2 - 1.5 |m|^2) / rho]
// and the moments M0 = sum t mu, M_a = sum t c_a mu, M_ab = sum t c_a c_b mu:
//   sum mu d_rho feq(rho, m) = M0 - (4.5 m.M2.m - 1.5 |m|^2 M0) / rho^2,
//   sum mu d_m   feq(rho, m) = 3 M1 + (9 M2.m - 3 m M0) / rho,
//   sum mu feq(rho, m)       = rho M0 + 3 m.M1 + (4.5 m.M2.m - 1.5 |m|^2 M0) / rho.
struct MuMoments {
  double m0, mx, my, mxx, mxy, myy;
};

__device__ __forceinline__ MuMoments mu_moments(const double (&mu)[kQ]) {
  constexpr double t1 = 1.0 / 9.0, t2 = 1.0 / 36.0;
  // sums and differences of the opposite pairs (1, 3), (2, 4), (5, 7), (6, 8)
  const double s13 = mu[1] + mu[3], d13 = mu[1] - mu[3], s24 = mu[2] + mu[4], d24 = mu[2] - mu[4];
  const double s57 = mu[5] + mu[7], d57 = mu[5] - mu[7], s68 = mu[6] + mu[8], d68 = mu[6] - mu[8];
  const double diag = s57 + s68;
  MuMoments M;
  M.m0 = fma(4.0 / 9.0, mu[0], fma(t1, s13 + s24, t2 * diag));
  M.mx = fma(t1, d13, t2 * (d57 - d68));
  M.my = fma(t1, d24, t2 * (d57 + d68));
  M.mxx = fma(t1, s13, t2 * diag);
  M.myy = fma(t1, s24, t2 * diag);
  M.mxy = t2 * (s57 - s68);
  return M;
}

// Adjoint of one step (see the header comment).  with_obj adds dJ_n/df on
// the objective region R.  Each CTA's (dJ/dtau, dJ/dF0) sums go to its slot
// of `partials`, added to what is there when `add` (a sweep's running sums;
// steps are stream-ordered, so a slot has one writer at a time).
__global__ void k_adjoint(AGrid g, Region R, const double *f, const double *lam_in,
                          double *lam_out, const double *F, int with_obj, double *partials,
                          int add) {
  double acc[2] = {0.0, 0.0};
  FOR_CELLS {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    double fl[kQ], mu[kQ];
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      fl[l] = f[(size_t)l * N + c];
      const int xd = wr(x + cx_of(l), g.nx), yd = wr(y + cy_of(l), g.ny);
      mu[l] = lam_in ? lam_in[(size_t)l * N + (size_t)yd * g.nx + xd] : 0.0;
    }
    // moments from the opposite pairs' sums and differences
    const double d57 = fl[5] - fl[7], d68 = fl[6] - fl[8];
    const double rho = fl[0] + ((fl[1] + fl[3]) + (fl[2] + fl[4])) + ((fl[5] + fl[7]) + (fl[6] + fl[8]));
    const double jx = (fl[1] - fl[3]) + (d57 - d68), jy = (fl[2] - fl[4]) + (d57 + d68);
    const double ir = 1.0 / rho;
    const double mpx = (1.0 - g.alpha) * jx + g.fxt[y];
    const double mpy = (1.0 - g.alpha) * jy + g.fyt[x];
    const MuMoments M = mu_moments(mu);
    // equilibrium at (rho, j): q_a = m.M2.m, p_a = M2.m
    const double pax = M.mxx * jx + M.mxy * jy, pay = M.mxy * jx + M.myy * jy;
    const double qa = (4.5 * (jx * pax + jy * pay) - 1.5 * (jx * jx + jy * jy) * M.m0) * ir;
    // at (rho, m')
    const double pbx = M.mxx * mpx + M.mxy * mpy, pby = M.mxy * mpx + M.myy * mpy;
    const double qb = (4.5 * (mpx * pbx + mpy * pby) - 1.5 * (mpx * mpx + mpy * mpy) * M.m0) * ir;
    const double w1 = g.omega - 1.0;
    const double Sa_rho = M.m0 - qa * ir, Sb_rho = M.m0 - qb * ir;
    // S_a = 3 M_a + 9 p_a / rho - 3 m_a M0 / rho with 9 / rho and 3 M0 / rho
    // formed once
    const double ir9 = 9.0 * ir, k0 = 3.0 * M.m0 * ir, mx3 = 3.0 * M.mx, my3 = 3.0 * M.my;
    const double Sa_x = fma(ir9, pax, fma(-jx, k0, mx3));
    const double Sa_y = fma(ir9, pay, fma(-jy, k0, my3));
    const double Sb_x = fma(ir9, pbx, fma(-mpx, k0, mx3));
    const double Sb_y = fma(ir9, pby, fma(-mpy, k0, my3));
    double Arho = w1 * Sa_rho + Sb_rho;
    double Ajx = w1 * Sa_x + (1.0 - g.alpha) * Sb_x;
    double Ajy = w1 * Sa_y + (1.0 - g.alpha) * Sb_y;
    // sum mu (f - feq(rho, j)) for dJ/dtau
    double muf = 0.0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) muf += mu[l] * fl[l];
    const double mufeq = rho * M.m0 + 3.0 * (jx * M.mx + jy * M.my) + qa;
    const double sx = F[S_TAB * N + y], sy = F[S_TAB * N + g.ny + x];
    acc[0] += (muf - mufeq) * g.omega * g.omega;  // / tau^2
    acc[1] += Sb_x * sx + Sb_y * sy;
    if (with_obj && in_region(x, y, R, g)) {
      Arho += F[D_TOT * N + c];
      Ajx += F[D_JX * N + c];
      Ajy += F[D_JY * N + c];
    }
    const double keep = 1.0 - g.omega;
    // lambda_l = keep mu_l + Arho + c_l . A, by opposite pairs (c . A once
    // per pair; a product by c = 0 still costs an FMA under IEEE arithmetic)
    const double cA[4] = {Ajx, Ajy, Ajx + Ajy, Ajy - Ajx};  // c of 1, 2, 5, 6
    lam_out[c] = fma(keep, mu[0], Arho);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int l = k < 2 ? 1 + k : 5 + (k - 2), m = opposite(l);
      lam_out[(size_t)l * N + c] = fma(keep, mu[l], Arho + cA[k]);
      lam_out[(size_t)m * N + c] = fma(keep, mu[m], Arho - cA[k]);
    }
  }
  block_sums<2>(acc, partials + 2 * blockIdx.x, add);
}

// Adds every partial into the two accumulators: thread i sums the partials
// i, i + 256, ... in order, then a fixed-order tree in shared memory (the
// same order every call: block-deterministic).
__global__ void __launch_bounds__(256) k_adjoint_final(const double *p_step, int nb,
                                                       const double *p_tau, int nbo,
                                                       const double *p_F0, int nbr, int with_obj,
                                                       double *dJ_dtau, double *dJ_dF0) {
  __shared__ double sa[256], sb[256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = t; i < nb; i += 256) {
    a += p_step[2 * i];
    b += p_step[2 * i + 1];
  }
  if (with_obj) {
    for (int i = t; i < nbo; i += 256) a += p_tau[i];
    for (int i = t; i < nbr; i += 256) b += p_F0[i];
  }
  sa[t] = a;
  sb[t] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) {
      sa[t] += sa[t + w];
      sb[t] += sb[t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    if (dJ_dtau) *dJ_dtau += sa[0];
    if (dJ_dF0) *dJ_dF0 += sb[0];
  }
}

// The forward objective in one launch of many CTAs.  The box is cut into
// TB x TB tiles; for each of its tiles a CTA computes rho and u = (j +
// F/2)/rho from the storage state `state` (the snapshot's moment arithmetic)
// on the tile widened by the 4-cell reach of the eq. (18) stencils (cells of
// the overlaps computed once per tile that needs them), keeps them in shared
// memory and sums the dissipation terms of the tile's box cells.  Each CTA
// writes one partial; the last CTA to finish (the arrival counter `count`,
// zero before the launch and reset by that CTA) sums the partials in a fixed
// order and adds cw times the sum to acc.  Small tiles for small boxes, a
// thread per cell of the widened tile and four lanes per box cell: the FP64
// work spreads over more SMs and its dependent chains stay short (GB300
// issues about 1.7 FP64 FMAs per clock per SM).
template <typename T, int TB, int NT>
__global__ void __launch_bounds__(NT)
    k_obj_tiles(const Member *__restrict__ members, int member, int state, AGrid g, int bx,
                int by, int L, double cw, double *partials, unsigned *count, double *acc) {
  constexpr int W = TB + 8, NC = W * W;
  __shared__ double sr[NC], su[NC], sv[NC];
  __shared__ double sw[NT / 32];
  __shared__ int is_last;
  const Member &M = members[member];
  const T *src = static_cast<const T *>(state_buffer(M, state));
  const int tid = threadIdx.x, ntx = (L + TB - 1) / TB, nt = ntx * ntx;
  double a = 0.0;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int ox = (t % ntx) * TB, oy = (t / ntx) * TB;  // tile origin within the box
    __syncthreads();  // the previous tile's reads of shared memory are done
    for (int i = tid; i < NC; i += NT) {
      const int x = wrapi(bx + ox - 4 + i % W, g.nx), y = wrapi(by + oy - 4 + i / W, g.ny);
      T f[kQ];
#pragma unroll
      for (int l = 0; l < kQ; ++l) f[l] = src[pub_index(M, state, l, x, y)];
      double r, jx, jy;
      pub_moments<T>(f, M.rho0, r, jx, jy);
      const double Fx = g.fxt[y] - g.alpha * jx, Fy = g.fyt[x] - g.alpha * jy;
      const double ir = 1.0 / r;
      sr[i] = r;
      su[i] = (jx + 0.5 * Fx) * ir;
      sv[i] = (jy + 0.5 * Fy) * ir;
    }
    __syncthreads();
    // the tile's box cells, four lanes per cell (d/dx u, d/dy u, d/dx v,
    // d/dy v), whole warps per pass so that every shuffle has the full warp
    const int lane = tid & 31, p = lane & 3, qb = lane & ~3;
    for (int i0 = (tid >> 5) * 8; i0 < TB * TB; i0 += (NT / 32) * 8) {
      const int iq = i0 + (lane >> 2), i = iq < TB * TB ? iq : TB * TB - 1;
      const int lx = i % TB, ly = i / TB;
      const int c = (ly + 4) * W + lx + 4, s = (p & 1) ? W : 1;
      const double *A = p < 2 ? su : sv;
      const double d = 0.8 * (A[c + s] - A[c - s]) - 0.2 * (A[c + 2 * s] - A[c - 2 * s]) +
                       (4.0 / 105.0) * (A[c + 3 * s] - A[c - 3 * s]) -
                       (1.0 / 280.0) * (A[c + 4 * s] - A[c - 4 * s]);
      const double dxu = __shfl_sync(0xffffffffu, d, qb), dyu = __shfl_sync(0xffffffffu, d, qb + 1);
      const double dxv = __shfl_sync(0xffffffffu, d, qb + 2), dyv = __shfl_sync(0xffffffffu, d, qb + 3);
      if (p == 0 && iq < TB * TB && ox + lx < L && oy + ly < L) {
        const double sxx = 2 * dxu, sxy = dyu + dxv, syy = 2 * dyv;
        a += -g.nu * sr[c] * (sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv);
      }
    }
  }
  // the CTA's partial: shuffle tree per warp, warps in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((tid & 31) == 0) sw[tid >> 5] = a;
  __syncthreads();
  if (tid == 0) {
    double p = 0.0;
    for (int w = 0; w < NT / 32; ++w) p += sw[w];
    partials[blockIdx.x] = p;
    __threadfence();
    is_last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // last CTA: strided fixed-order chains, the same tree
  double b = 0.0;
  for (int k = tid; k < (int)gridDim.x; k += NT) b += __ldcg(partials + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
  __syncthreads();
  if ((tid & 31) == 0) sw[tid >> 5] = b;
  __syncthreads();
  if (tid == 0) {
    double p = 0.0;
    for (int w = 0; w < NT / 32; ++w) p += sw[w];
    *acc += cw * p;
    *count = 0u;
  }
}

template <typename T>
cudaError_t launch_obj_tiles(const Member *d_members, int member, int state, const AGrid &g,
                             int bx, int by, int L, double cw, double *partials,
                             unsigned *count, double *acc, cudaStream_t s) {
  // the largest tile that still gives a CTA to every SM, 4 x 4 at least;
  // a thread per cell of the widened tile ((TB + 8)^2 rounded up to warps)
  // for the latency-bound small tiles, 256 threads for 16 x 16 tiles, whose
  // many CTAs keep the FP64 pipes busy (L = 256 on 256^2: 28.8 us against
  // 30.8 with 576 threads)
  auto tiles = [&](int tb) { return (long long)((L + tb - 1) / tb) * ((L + tb - 1) / tb); };
  const int tb = tiles(16) >= 152 ? 16 : tiles(8) >= 152 ? 8 : 4;
  const int grid = (int)std::min<long long>(tiles(tb), kMaxPartialBlocks);
  if (tb == 16)
    k_obj_tiles<T, 16, 256><<<grid, 256, 0, s>>>(d_members, member, state, g, bx, by, L, cw,
                                                 partials, count, acc);
  else if (tb == 8)
    k_obj_tiles<T, 8, 256><<<grid, 256, 0, s>>>(d_members, member, state, g, bx, by, L, cw,
                                                partials, count, acc);
  else
    k_obj_tiles<T, 4, 160><<<grid, 160, 0, s>>>(d_members, member, state, g, bx, by, L, cw,
                                                partials, count, acc);
  return cudaGetLastError();
}

AGrid agrid(const Member &hm) {
  AGrid g;
  g.nx = hm.nx;
  g.ny = hm.ny;
  g.kf = hm.kf;
  g.force = hm.force_kind;
  g.nu = hm.nu;
  g.alpha = hm.alpha;
  g.tau = hm.tau;
  g.omega = hm.omega;
  g.F0 = hm.F0;
  g.fxt = hm.fx_tab64;
  g.fyt = hm.fy_tab64;
  return g;
}

int nblocks_for(size_t N, int threads = 256) {
  size_t b = (N + threads - 1) / threads;
  return (int)(b > (size_t)kMaxPartialBlocks ? kMaxPartialBlocks : (b < 1 ? 1 : b));
}

// CTA size of the objective kernels of an adjoint step: their few hundred
// to few thousand cells of FP64 work spread over as many SMs as possible
// (GB300 issues about 1.7 FP64 FMAs per clock per SM).  A 100-level sweep
// of 256^2 with every other level weighted (L = 16): 42.8 us per level with
// 32-thread CTAs, 44.4 with 256 threads, 52.0 with the three kernels in one
// single-CTA launch.
constexpr int kObjThreads = 32;

// CTA size of k_adjoint: 64 threads below 2^17 cells, so that a small
// grid's FP64 work spreads evenly over the SMs (256^2: 44.3 against 46.2 us
// per adjoint step with 256-thread CTAs in 1.7 waves), 256 above.
int adjoint_threads(size_t N) { return N < ((size_t)1 << 17) ? 64 : 256; }

}  // namespace

cudaError_t adjoint_step(const Member &hm, const double *f_n, const double *lam_in,
                         double *lam_out, double w, int bx, int by, int L, double *dJ_dtau,
                         double *dJ_dF0, const DiagScratch &sc, cudaStream_t s) {
  const AGrid g = agrid(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  const int tpb = adjoint_threads(N), nb = nblocks_for(N, tpb);
  double *F = sc.f;
  double *p_step = sc.partials;                         // [nb][2]
  double *p_tau = p_step + 2 * kMaxPartialBlocks;       // [nbo]
  double *p_F0 = p_tau + kMaxPartialBlocks;             // [nbr]
  const int with_obj = w != 0.0;
  const Region R = objective_region(hm.nx, hm.ny, bx, by, L);
  int nbo = 0, nbr = 0;
  k_sine_tables<<<(hm.nx + hm.ny + 255) / 256, 256, 0, s>>>(g, F + S_TAB * N);
  if (with_obj) {
    const double cw = w / ((double)L * (double)L);
    const size_t nreg = (size_t)R.w * R.h;
    nbr = nblocks_for(4 * nreg, kObjThreads);  // four lanes per cell
    nbo = nblocks_for(4 * (size_t)L * L, kObjThreads);
    k_region_velocity<<<nblocks_for(nreg, kObjThreads), kObjThreads, 0, s>>>(g, R, f_n, F);
    k_obj_gamma<<<nbo, kObjThreads, 0, s>>>(g, F, cw, bx, by, L, p_tau, 0);
    k_obj_velocity_adjoint<<<nbr, kObjThreads, 0, s>>>(g, R, F, bx, by, L, p_F0, 0);
  }
  k_adjoint<<<nb, tpb, 0, s>>>(g, R, f_n, lam_in, lam_out, F, with_obj, p_step, 0);
  k_adjoint_final<<<1, 256, 0, s>>>(p_step, nb, p_tau, nbo, p_F0, nbr, with_obj, dJ_dtau,
                                    dJ_dF0);
  return cudaGetLastError();
}

int adjoint_kernel_count(double w) { return w != 0.0 ? 6 : 3; }

// The adjoint steps of states[nstates - 1] .. states[0] (each [9][ny][nx]),
// the adjoint ping-ponging between lam_out and lam_tmp so that the last
// (state 0) lands in lam_out; weights[k] (host) the objective weight of
// step k.  Each CTA keeps running sums of its (dJ/dtau, dJ/dF0) partials
// over the whole sweep and one reduction at the end adds them into the
// accumulators; the force-direction tables are built once.  The adjoint
// fields are those of per-step adjoint_step calls; the two gradients differ
// from theirs only by the order of the FP64 sums.
cudaError_t adjoint_sweep(const Member &hm, const double *states, int nstates,
                          const double *lam_in, double *lam_out, double *lam_tmp,
                          const double *weights, int bx, int by, int L, double *dJ_dtau,
                          double *dJ_dF0, const DiagScratch &sc, cudaStream_t s,
                          long long *launches) {
  const AGrid g = agrid(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  const int tpb = adjoint_threads(N), nb = nblocks_for(N, tpb);
  double *F = sc.f;
  double *p_step = sc.partials;                    // [nb][2]
  double *p_tau = p_step + 2 * kMaxPartialBlocks;  // [nbo]
  double *p_F0 = p_tau + kMaxPartialBlocks;        // [nbr]
  int any_obj = 0;
  for (int k = 0; k < nstates; ++k) any_obj |= weights[k] != 0.0;
  const Region R = objective_region(hm.nx, hm.ny, bx, by, L);
  const size_t nreg = (size_t)R.w * R.h;
  const int nbv = nblocks_for(nreg, kObjThreads);
  const int nbr = any_obj ? nblocks_for(4 * nreg, kObjThreads) : 0;  // four lanes per cell
  const int nbo = any_obj ? nblocks_for(4 * (size_t)L * L, kObjThreads) : 0;
  cudaError_t e = cudaMemsetAsync(p_step, 0, sizeof(double) * 4 * kMaxPartialBlocks, s);
  if (e != cudaSuccess) return e;
  k_sine_tables<<<(hm.nx + hm.ny + 255) / 256, 256, 0, s>>>(g, F + S_TAB * N);
  long long n = 2;
  const double *in = lam_in;
  for (int k = nstates - 1; k >= 0; --k) {
    double *out = (k % 2 == 0) ? lam_out : lam_tmp;
    const double *f_k = states + (size_t)k * kQ * N;
    const int with_obj = weights[k] != 0.0;
    if (with_obj) {
      const double cw = weights[k] / ((double)L * (double)L);
      k_region_velocity<<<nbv, kObjThreads, 0, s>>>(g, R, f_k, F);
      k_obj_gamma<<<nbo, kObjThreads, 0, s>>>(g, F, cw, bx, by, L, p_tau, 1);
      k_obj_velocity_adjoint<<<nbr, kObjThreads, 0, s>>>(g, R, F, bx, by, L, p_F0, 1);
      n += 3;
    }
    k_adjoint<<<nb, tpb, 0, s>>>(g, R, f_k, in, out, F, with_obj, p_step, 1);
    n += 1;
    in = out;
  }
  k_adjoint_final<<<1, 256, 0, s>>>(p_step, nb, p_tau, nbo, p_F0, nbr, any_obj, dJ_dtau, dJ_dF0);
  if (launches) *launches += n;
  return cudaGetLastError();
}

// Forward objective of the state in storage `state`: one launch.
cudaError_t objective_tiles(int precision, const Member *d_members, int member,
                            const Member &hm, int state, double w, int bx, int by, int L,
                            double *acc, const DiagScratch &sc, cudaStream_t s) {
  const AGrid g = agrid(hm);
  const double cw = w / ((double)L * (double)L);
  if (precision == 32)
    return launch_obj_tiles<float>(d_members, member, state, g, bx, by, L, cw, sc.partials,
                                   sc.count, acc, s);
  return launch_obj_tiles<double>(d_members, member, state, g, bx, by, L, cw, sc.partials,
                                  sc.count, acc, s);
}

}  // namespace lbm
