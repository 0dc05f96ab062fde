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
#include "lbm_internal.cuh"

namespace lbm {

namespace {

enum AdjField { A_RHO = 0, A_JX, A_JY, A_U, A_V, GAM_XX, GAM_XY, GAM_YY, D_RHO, D_JX, D_JY,
                A_NFIELDS };
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

__device__ __forceinline__ double Dx(const double *A, const AGrid &g, int x, int y) {
  const double *r = A + (size_t)y * g.nx;
  return 0.8 * (r[wr(x + 1, g.nx)] - r[wr(x - 1, g.nx)]) -
         0.2 * (r[wr(x + 2, g.nx)] - r[wr(x - 2, g.nx)]) +
         (4.0 / 105.0) * (r[wr(x + 3, g.nx)] - r[wr(x - 3, g.nx)]) -
         (1.0 / 280.0) * (r[wr(x + 4, g.nx)] - r[wr(x - 4, g.nx)]);
}
__device__ __forceinline__ double Dy(const double *A, const AGrid &g, int x, int y) {
  auto at = [&](int d) { return A[(size_t)wr(y + d, g.ny) * g.nx + x]; };
  return 0.8 * (at(1) - at(-1)) - 0.2 * (at(2) - at(-2)) + (4.0 / 105.0) * (at(3) - at(-3)) -
         (1.0 / 280.0) * (at(4) - at(-4));
}

__device__ __forceinline__ bool in_box(int x, int y, int bx, int by, int L, const AGrid &g) {
  return wrapi(x - bx, g.nx) < L && wrapi(y - by, g.ny) < L;
}

__device__ __forceinline__ void force_dir(const AGrid &g, int x, int y, double &sx, double &sy) {
  if (g.force == 1) {
    sx = sinpi(2.0 * g.kf * (double)y / g.ny);
    sy = sinpi(2.0 * g.kf * (double)x / g.nx);
  } else {
    sx = 0.0;
    sy = 0.0;
  }
}

template <int NQ>
__device__ void block_sums(double (&v)[NQ], double *out) {
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
    out[tid] = a;
  }
}

#define FOR_CELLS                                                                   \
  const size_t N = (size_t)g.nx * g.ny;                                             \
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;             \
       c += (size_t)gridDim.x * blockDim.x)

// rho and j of the public state f[9][ny][nx].
__global__ void k_public_moments(AGrid g, const double *f, double *F) {
  FOR_CELLS {
    double r = 0, a = 0, b = 0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const double v = f[(size_t)l * N + c];
      r += v;
      a += cx_of(l) * v;
      b += cy_of(l) * v;
    }
    F[A_RHO * N + c] = r;
    F[A_JX * N + c] = a;
    F[A_JY * N + c] = b;
  }
}

// u = (j + F/2)/rho from (rho, j) fields at F + 0..2N.
__global__ void k_velocity(AGrid g, double *F) {
  FOR_CELLS {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    const double r = F[A_RHO * N + c], jx = F[A_JX * N + c], jy = F[A_JY * N + c];
    const double Fx = g.fxt[y] - g.alpha * jx, Fy = g.fyt[x] - g.alpha * jy;
    F[A_U * N + c] = (jx + 0.5 * Fx) / r;
    F[A_V * N + c] = (jy + 0.5 * Fy) / r;
  }
}

// Objective pass 1: Gamma_ij = dJ/dG_ij = -2 c nu rho S_ij in the box
// (c = weight / L^2); direct rho part -c nu Q; explicit dJ/dtau part.
__global__ void k_obj_gamma(AGrid g, double *F, double cw, int bx, int by, int L,
                            double *partials) {
  double acc[1] = {0.0};
  FOR_CELLS {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    double gxx = 0, gxy = 0, gyy = 0, drho = 0;
    if (in_box(x, y, bx, by, L, g)) {
      const double *U = F + A_U * N, *V = F + A_V * N;
      const double dxu = Dx(U, g, x, y), dyu = Dy(U, g, x, y);
      const double dxv = Dx(V, g, x, y), dyv = Dy(V, g, x, y);
      const double sxx = 2 * dxu, sxy = dyu + dxv, syy = 2 * dyv;
      const double Q = sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv;
      const double r = F[A_RHO * N + c];
      gxx = -2.0 * cw * g.nu * r * sxx;
      gxy = -2.0 * cw * g.nu * r * sxy;
      gyy = -2.0 * cw * g.nu * r * syy;
      drho = -cw * g.nu * Q;
      acc[0] += -cw * r * Q / 3.0;  // d nu / d tau = 1/3
    }
    F[GAM_XX * N + c] = gxx;
    F[GAM_XY * N + c] = gxy;
    F[GAM_YY * N + c] = gyy;
    F[D_RHO * N + c] = drho;
  }
  block_sums<1>(acc, partials + blockIdx.x);
}

// Objective pass 2: dJ/du_i = -sum_j D_j Gamma_ij, then dJ/drho, dJ/dj and
// the explicit dJ/dF0 part through u = ((1 - alpha/2) j + F_ext/2)/rho.
__global__ void k_obj_velocity_adjoint(AGrid g, double *F, double *partials) {
  double acc[1] = {0.0};
  FOR_CELLS {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    const double Ux = -(Dx(F + GAM_XX * N, g, x, y) + Dy(F + GAM_XY * N, g, x, y));
    const double Uy = -(Dx(F + GAM_XY * N, g, x, y) + Dy(F + GAM_YY * N, g, x, y));
    const double r = F[A_RHO * N + c], u = F[A_U * N + c], v = F[A_V * N + c];
    F[D_RHO * N + c] += -(Ux * u + Uy * v) / r;
    F[D_JX * N + c] = Ux * (1.0 - 0.5 * g.alpha) / r;
    F[D_JY * N + c] = Uy * (1.0 - 0.5 * g.alpha) / r;
    double sx, sy;
    force_dir(g, x, y, sx, sy);
    acc[0] += (Ux * sx + Uy * sy) / (2.0 * r);
  }
  block_sums<1>(acc, partials + blockIdx.x);
}

// Adjoint of one step (see the header comment).  with_obj adds dJ_n/df.
__global__ void k_adjoint(AGrid g, const double *f, const double *lam_in, double *lam_out,
                          const double *F, int with_obj, double *partials) {
  double acc[2] = {0.0, 0.0};
  FOR_CELLS {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    double fl[kQ], mu[kQ];
    double rho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      fl[l] = f[(size_t)l * N + c];
      rho += fl[l];
      jx += cx_of(l) * fl[l];
      jy += cy_of(l) * fl[l];
      const int xd = wr(x + cx_of(l), g.nx), yd = wr(y + cy_of(l), g.ny);
      mu[l] = lam_in ? lam_in[(size_t)l * N + (size_t)yd * g.nx + xd] : 0.0;
    }
    const double ir = 1.0 / rho;
    const double mpx = (1.0 - g.alpha) * jx + g.fxt[y];
    const double mpy = (1.0 - g.alpha) * jy + g.fyt[x];
    const double jj = jx * jx + jy * jy, mm = mpx * mpx + mpy * mpy;
    double sx, sy;
    force_dir(g, x, y, sx, sy);
    const double w1 = g.omega - 1.0;
    double Arho = 0, Ajx = 0, Ajy = 0, dtau = 0, dF0 = 0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const double t = w_of(l);
      const double cxl = cx_of(l), cyl = cy_of(l);
      const double cj = cxl * jx + cyl * jy, cm = cxl * mpx + cyl * mpy;
      // equilibrium at (rho, j) and its derivatives
      const double feq = t * (rho + 3.0 * cj + (4.5 * cj * cj - 1.5 * jj) * ir);
      const double drho_a = t * (1.0 - (4.5 * cj * cj - 1.5 * jj) * ir * ir);
      const double dmx_a = t * (3.0 * cxl + (9.0 * cj * cxl - 3.0 * jx) * ir);
      const double dmy_a = t * (3.0 * cyl + (9.0 * cj * cyl - 3.0 * jy) * ir);
      // at (rho, m')
      const double drho_b = t * (1.0 - (4.5 * cm * cm - 1.5 * mm) * ir * ir);
      const double dmx_b = t * (3.0 * cxl + (9.0 * cm * cxl - 3.0 * mpx) * ir);
      const double dmy_b = t * (3.0 * cyl + (9.0 * cm * cyl - 3.0 * mpy) * ir);
      const double m = mu[l];
      Arho += m * (w1 * drho_a + drho_b);
      Ajx += m * (w1 * dmx_a + (1.0 - g.alpha) * dmx_b);
      Ajy += m * (w1 * dmy_a + (1.0 - g.alpha) * dmy_b);
      dtau += m * (fl[l] - feq);
      dF0 += m * (dmx_b * sx + dmy_b * sy);
    }
    double orho = 0, ojx = 0, ojy = 0;
    if (with_obj) {
      orho = F[D_RHO * N + c];
      ojx = F[D_JX * N + c];
      ojy = F[D_JY * N + c];
    }
#pragma unroll
    for (int l = 0; l < kQ; ++l)
      lam_out[(size_t)l * N + c] = (1.0 - g.omega) * mu[l] + Arho + cx_of(l) * Ajx +
                                   cy_of(l) * Ajy + orho + cx_of(l) * ojx + cy_of(l) * ojy;
    acc[0] += dtau / (g.tau * g.tau);
    acc[1] += dF0;
  }
  block_sums<2>(acc, partials + 2 * blockIdx.x);
}

// Adds every partial, in block order, into the two accumulators.
__global__ void k_adjoint_final(const double *p_step, int nb, const double *p_tau,
                                const double *p_F0, int nbo, int with_obj, double *dJ_dtau,
                                double *dJ_dF0) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) {
    a += p_step[2 * i];
    b += p_step[2 * i + 1];
  }
  if (with_obj)
    for (int i = 0; i < nbo; ++i) {
      a += p_tau[i];
      b += p_F0[i];
    }
  if (dJ_dtau) *dJ_dtau += a;
  if (dJ_dF0) *dJ_dF0 += b;
}

// Forward objective on (rho, j): acc += weight / L^2 * sum_box eps.
__global__ void k_obj_forward(AGrid g, const double *F, double cw, int bx, int by, int L,
                              double *partials) {
  double acc[1] = {0.0};
  const size_t nbox = (size_t)L * L;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nbox;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = wrapi(bx + (int)(i % L), g.nx), y = wrapi(by + (int)(i / L), g.ny);
    const size_t N = (size_t)g.nx * g.ny, c = (size_t)y * g.nx + x;
    const double *U = F + A_U * N, *V = F + A_V * N;
    const double dxu = Dx(U, g, x, y), dyu = Dy(U, g, x, y);
    const double dxv = Dx(V, g, x, y), dyv = Dy(V, g, x, y);
    const double sxx = 2 * dxu, sxy = dyu + dxv, syy = 2 * dyv;
    acc[0] += -g.nu * F[A_RHO * N + c] * (sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv);
  }
  block_sums<1>(acc, partials + blockIdx.x);
}

__global__ void k_obj_forward_final(const double *partials, int nb, double cw, double *acc) {
  if (threadIdx.x != 0) return;
  double a = 0.0;
  for (int i = 0; i < nb; ++i) a += partials[i];
  *acc += cw * a;
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

int nblocks_for(size_t N) {
  size_t b = (N + 255) / 256;
  return (int)(b > (size_t)kMaxPartialBlocks ? kMaxPartialBlocks : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t adjoint_step(const Member &hm, const double *f_n, const double *lam_in,
                         double *lam_out, double w, int bx, int by, int L, double *dJ_dtau,
                         double *dJ_dF0, const DiagScratch &sc, cudaStream_t s) {
  const AGrid g = agrid(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  const int nb = nblocks_for(N);
  double *F = sc.f;
  double *p_step = sc.partials;                         // [nb][2]
  double *p_tau = p_step + 2 * kMaxPartialBlocks;       // [nb]
  double *p_F0 = p_tau + kMaxPartialBlocks;             // [nb]
  const int with_obj = w != 0.0;
  if (with_obj) {
    const double cw = w / ((double)L * (double)L);
    k_public_moments<<<nb, 256, 0, s>>>(g, f_n, F);
    k_velocity<<<nb, 256, 0, s>>>(g, F);
    k_obj_gamma<<<nb, 256, 0, s>>>(g, F, cw, bx, by, L, p_tau);
    k_obj_velocity_adjoint<<<nb, 256, 0, s>>>(g, F, p_F0);
  }
  k_adjoint<<<nb, 256, 0, s>>>(g, f_n, lam_in, lam_out, F, with_obj, p_step);
  k_adjoint_final<<<1, 32, 0, s>>>(p_step, nb, p_tau, p_F0, nb, with_obj, dJ_dtau, dJ_dF0);
  return cudaGetLastError();
}

int adjoint_kernel_count(double w) { return w != 0.0 ? 6 : 2; }

// Forward objective from the (rho, j) snapshot already written to sc.f[0..2].
cudaError_t objective_from_snapshot(const Member &hm, double w, int bx, int by, int L,
                                    double *acc, const DiagScratch &sc, cudaStream_t s) {
  const AGrid g = agrid(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  double *F = sc.f;
  k_velocity<<<nblocks_for(N), 256, 0, s>>>(g, F);
  const int nb = nblocks_for((size_t)L * L);
  k_obj_forward<<<nb, 256, 0, s>>>(g, F, 0.0, bx, by, L, sc.partials);
  k_obj_forward_final<<<1, 32, 0, s>>>(sc.partials, nb, w / ((double)L * (double)L), acc);
  return cudaGetLastError();
}

}  // namespace lbm
