/*
 * Oracle for the D2Q9 LBGK method and the sub-volume energy/enstrophy
 * balance diagnostic of Tauzin, Biferale, Sbragaglia, Gupta, Toschi,
 * Bartel, Ehrhardt, "A numerical tool for the study of the hydrodynamic
 * recovery of the Lattice Boltzmann Method", Comput. & Fluids 172 (2018).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64, single
 * threaded CPU restatement of the method, written so that each function can
 * be checked against the paper by eye.  It shares no code, header, table or
 * constant with the CUDA library; only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  Nothing in the product
 * path calls it.
 *
 * Conventions (the paper leaves these open; every reading is listed in the
 * design notes of the repository):
 *   - Lattice order: c_0=(0,0); c_1..c_4=(1,0),(0,1),(-1,0),(0,-1);
 *     c_5..c_8=(1,1),(-1,1),(-1,-1),(1,-1).  Weights 4/9, 1/9, 1/36, and
 *     c_s^2 = 1/3 (the standard D2Q9 of the paper's Sec. 3).
 *   - Arrays are row-major: f[(l*ny + y)*nx + x], fields A[y*nx + x];
 *     x is the first (i) index of the paper's eq. (18), y the second (j).
 *   - The state f(x, n) is the pre-collision population of eq. (1).
 *   - Forcing: Kolmogorov body force F_ext = F0 (sin(2 pi kf y/ny),
 *     sin(2 pi kf x/nx)) plus linear drag -alpha j on the bare momentum,
 *     applied with the exact-difference method (EDM) the paper names in
 *     Sec. 3: F_l = f_eq(rho, u + F/rho) - f_eq(rho, u).
 *   - Diagnostic velocity: u_phys = (j + F/2)/rho.
 *   - Sub-volume averages wrap periodically; boxes are L x L with lower-left
 *     origin (x0, y0).
 *
 * Parity status: every function here is pinned by a CPU test (moment
 * identities, conservation, streaming permutation, Taylor-Green decay,
 * Kolmogorov laminar amplitude, stencil modified wavenumber, BDF2
 * exactness, symbolic continuum terms, brute-force box sums, closed-form
 * box Mach numbers, brute-force histogram counts; the diagnostic velocity
 * by the midpoint of the momenta before and after the force acts; the ELBM
 * relaxation by a near-equilibrium shear-wave decay at the BGK viscosity
 * and by the per-cell relaxation at the tau_eff of its local viscosity).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 9
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double TW[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;
static const double PI = 3.14159265358979323846;

/* Model of one member.  Forcing (Sec. 3 and the workloads):
 *   kind 0: none;
 *   kind 1: Kolmogorov F_ext = F0 (sin(2 pi kf y/ny), sin(2 pi kf x/nx));
 *   kind 2: the paper's turbulence forcing, the shell force of eqs. (14),
 *           (15) with amplitude F0 = F^T_0 and phase `phase`, plus the
 *           large-scale damping of eq. (16) with amplitude FR0 = F^R_0;
 * and in every case the linear drag -alpha j on the bare momentum.
 * Collision (Sec. 1): 0 BGK with tau; 1 Smagorinsky eddy viscosity
 * nu_t = C |S| (the paper's form, C = Cs, dx = 1); 2 the turbulent
 * viscosity of eq. (7); each gives a local tau_eff (orc_tau_eff); 3 the
 * entropic LBM (ELBM, orc_elbm_cell). */
typedef struct {
  int kind;
  double F0;
  int kf;
  double alpha;
  double phase;
  double FR0;
  int collision;
  double Cs;
} orc_model_t;

static int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------ */
/* Lattice                                                                  */
/* ------------------------------------------------------------------------ */

/* Copies the lattice tables out (for tests). */
void orc_lattice(int *cx, int *cy, double *t) {
  for (int l = 0; l < Q; ++l) {
    cx[l] = CX[l];
    cy[l] = CY[l];
    t[l] = TW[l];
  }
}

/* Equilibrium, eq. (2):
 *   f_eq_l = t_l rho [1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u.u/(2 cs^2)]. */
void orc_feq(double rho, double ux, double uy, double *feq) {
  double uu = ux * ux + uy * uy;
  for (int l = 0; l < Q; ++l) {
    double cu = CX[l] * ux + CY[l] * uy;
    feq[l] = TW[l] * rho *
             (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
  }
}

/* Time-independent external body force at cell (x, y): the Kolmogorov
 * force F0 (sin(2 pi kf y / ny), sin(2 pi kf x / nx)) for kind 1; for kind 2
 * the shell force of eqs. (14), (15),
 *   psi(x) = F^T_0 sum_k cos(2 pi (kx x / nx + ky y / ny) + phi),
 *   F^T = (d_y psi, -d_x psi)  (exact derivatives of each cosine),
 * the sum over one wavevector of each pair +-k with 5 <= |k| <= 7 (ky > 0,
 * or ky = 0 and kx > 0; over both members of each pair the phase would only
 * rescale the amplitude by 2 cos phi); zero otherwise. */
void orc_force_ext(int nx, int ny, const orc_model_t *F, int x, int y,
                   double *Fx, double *Fy) {
  *Fx = 0.0;
  *Fy = 0.0;
  if (F->kind == 1) {
    *Fx = F->F0 * sin(2.0 * PI * F->kf * (double)y / (double)ny);
    *Fy = F->F0 * sin(2.0 * PI * F->kf * (double)x / (double)nx);
  } else if (F->kind == 2) {
    double fx = 0.0, fy = 0.0;
    for (int ky = 0; ky <= 7; ++ky)
      for (int kx = -7; kx <= 7; ++kx) {
        int k2 = kx * kx + ky * ky;
        if (k2 < 25 || k2 > 49) continue;
        if (ky == 0 && kx <= 0) continue;
        double th = 2.0 * PI * (kx * (double)x / nx + ky * (double)y / ny) + F->phase;
        /* d_y cos(th) = -sin(th) 2 pi ky / ny; -d_x cos(th) = sin(th) 2 pi kx / nx */
        fx -= sin(th) * 2.0 * PI * ky / ny;
        fy += sin(th) * 2.0 * PI * kx / nx;
      }
    *Fx = F->F0 * fx;
    *Fy = F->F0 * fy;
  }
}

/* Large-scale damping of eq. (16) for the state f (kind 2):
 *   F^R(x) = -F^R_0 sum_{1 <= |k| <= 2} u^(k) exp(2 pi i (kx x / nx + ky y / ny)),
 *   u^(k) = (1 / (nx ny)) sum_x u(x) exp(-2 pi i (kx x / nx + ky y / ny)),
 * over the 12 wavevectors of the shell, u = j / rho the bare velocity of f.
 * With u^(k) = C_k - i S_k (C, S the cosine and sine sums over N) the
 * real part of each term is C_k cos(th) + S_k sin(th). */
static void damping_field(int nx, int ny, double FR0, const double *f,
                          double *FRx, double *FRy) {
  size_t N = (size_t)nx * ny;
  double *u = (double *)malloc(sizeof(double) * 2 * N);
  if (!u) return;
  for (size_t c = 0; c < N; ++c) {
    double r = 0.0, a = 0.0, b = 0.0;
    for (int l = 0; l < Q; ++l) {
      r += f[l * N + c];
      a += CX[l] * f[l * N + c];
      b += CY[l] * f[l * N + c];
    }
    u[c] = a / r;
    u[N + c] = b / r;
  }
  for (size_t c = 0; c < N; ++c) FRx[c] = FRy[c] = 0.0;
  for (int ky = -2; ky <= 2; ++ky)
    for (int kx = -2; kx <= 2; ++kx) {
      int k2 = kx * kx + ky * ky;
      if (k2 < 1 || k2 > 4) continue;
      double Cx = 0.0, Sx = 0.0, Cy = 0.0, Sy = 0.0;
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          size_t c = (size_t)y * nx + x;
          double th = 2.0 * PI * (kx * (double)x / nx + ky * (double)y / ny);
          Cx += u[c] * cos(th);
          Sx += u[c] * sin(th);
          Cy += u[N + c] * cos(th);
          Sy += u[N + c] * sin(th);
        }
      Cx /= (double)N;
      Sx /= (double)N;
      Cy /= (double)N;
      Sy /= (double)N;
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          size_t c = (size_t)y * nx + x;
          double th = 2.0 * PI * (kx * (double)x / nx + ky * (double)y / ny);
          FRx[c] -= FR0 * (Cx * cos(th) + Sx * sin(th));
          FRy[c] -= FR0 * (Cy * cos(th) + Sy * sin(th));
        }
    }
  free(u);
}

/* External force of every cell for the state f (drag excluded):
 * orc_force_ext plus, for kind 2, the damping of eq. (16). */
void orc_force_field(int nx, int ny, const orc_model_t *F, const double *f,
                     double *Fx, double *Fy) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x)
      orc_force_ext(nx, ny, F, x, y, &Fx[(size_t)y * nx + x], &Fy[(size_t)y * nx + x]);
  if (F->kind == 2 && F->FR0 != 0.0) {
    size_t N = (size_t)nx * ny;
    double *d = (double *)malloc(sizeof(double) * 2 * N);
    if (!d) return;
    damping_field(nx, ny, F->FR0, f, d, d + N);
    for (size_t c = 0; c < N; ++c) {
      Fx[c] += d[c];
      Fy[c] += d[N + c];
    }
    free(d);
  }
}

/* Moments below eq. (2): rho = sum_l f_l, j = sum_l c_l f_l (bare momentum,
 * u = j / rho). */
static void cell_moments(const double *fc, double *rho, double *jx,
                         double *jy) {
  double r = 0.0, a = 0.0, b = 0.0;
  for (int l = 0; l < Q; ++l) {
    r += fc[l];
    a += CX[l] * fc[l];
    b += CY[l] * fc[l];
  }
  *rho = r;
  *jx = a;
  *jy = b;
}

/* Collision of one cell: right-hand side of eq. (1) with the BGK operator
 * and the EDM forcing term.  fin/fout hold the 9 populations of the cell.
 * Total force F = F_ext - alpha j. */
void orc_collide_cell(const double *fin, double tau, double Fex, double Fey,
                      double alpha, double *fout) {
  double rho, jx, jy;
  cell_moments(fin, &rho, &jx, &jy);
  double ux = jx / rho, uy = jy / rho;
  double Fx = Fex - alpha * jx, Fy = Fey - alpha * jy;
  double feq[Q], feq_shift[Q];
  orc_feq(rho, ux, uy, feq);
  orc_feq(rho, ux + Fx / rho, uy + Fy / rho, feq_shift); /* EDM: u + F dt/rho */
  for (int l = 0; l < Q; ++l) {
    double Fl = feq_shift[l] - feq[l];
    fout[l] = fin[l] - (fin[l] - feq[l]) / tau + Fl;
  }
}

/* ------------------------------------------------------------------------ */
/* Entropic LBM (Sec. 1)                                                    */
/* ------------------------------------------------------------------------ */

/* The equilibrium of the entropic LBM: the minimiser of the H-function
 * H(f) = sum_l f_l ln(f_l / t_l) (Sec. 1) under fixed rho and j, which for
 * D2Q9 has the closed product form
 *   f_eq_l = t_l rho prod_{a = x, y} (2 - s_a) ((2 u_a + s_a) / (1 - u_a))^{c_la},
 *   s_a = sqrt(1 + 3 u_a^2). */
void orc_feq_entropic(double rho, double ux, double uy, double *feq) {
  double sx = sqrt(1.0 + 3.0 * ux * ux), sy = sqrt(1.0 + 3.0 * uy * uy);
  double bx = (2.0 * ux + sx) / (1.0 - ux), by = (2.0 * uy + sy) / (1.0 - uy);
  for (int l = 0; l < Q; ++l)
    feq[l] = TW[l] * rho * (2.0 - sx) * (2.0 - sy) * pow(bx, CX[l]) * pow(by, CY[l]);
}

/* phi(z) = (1 + z) ln(1 + z) - z, z > -1: a series for small |z| (where the
 * two terms cancel), else directly. */
static double phi_entropy(double z) {
  if (fabs(z) < 0.1) {
    double s = 0.0, p = z * z; /* sum_{k >= 2} (-1)^k z^k / (k (k - 1)) */
    for (int k = 2; k < 24; ++k) {
      s += ((k & 1) ? -p : p) / (double)(k * (k - 1));
      p *= z;
    }
    return s;
  }
  return (1.0 + z) * log1p(z) - z;
}

/* Entropy condition of ELBM for populations f and Delta = f_eq - f:
 *   g(a) = H(f + a Delta) - H(f)
 *        = sum_l f_l phi(a y_l) - a sum_l Delta_l ln(1 + y_l),  y = Delta / f,
 * an identity that uses sum_l Delta_l = 0 (mass) and keeps every term of the
 * difference of order Delta^2 (no cancellation of O(1) entropies). */
static double entropy_gap(const double *f, const double *d, double a) {
  double s1 = 0.0, s2 = 0.0;
  for (int l = 0; l < Q; ++l) {
    double y = d[l] / f[l];
    s1 += f[l] * phi_entropy(a * y);
    s2 += d[l] * log1p(y);
  }
  return s1 - a * s2;
}

/* The non-trivial root alpha > 1 of the entropy condition (g(0) = 0,
 * g(1) = H(f_eq) - H(f) <= 0, g convex): bisection on [1, a_max) where
 * a_max keeps every f_l + a Delta_l positive; alpha = 2 (the BGK value)
 * when the state is at equilibrium to rounding, when a population is not
 * positive, or when no root lies below min(a_max, 64). */
double orc_elbm_alpha(const double *f, const double *d) {
  double ymax = 0.0, amax = 64.0;
  for (int l = 0; l < Q; ++l) {
    if (!(f[l] > 0.0)) return 2.0;
    double y = d[l] / f[l];
    if (fabs(y) > ymax) ymax = fabs(y);
    if (y < 0.0 && -1.0 / y < amax) amax = -1.0 / y;
  }
  if (ymax < 1e-12) return 2.0;
  double lo = 1.0, hi = amax * (1.0 - 1e-12);
  if (entropy_gap(f, d, hi) < 0.0) return 2.0;
  for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
    double mid = 0.5 * (lo + hi);
    if (entropy_gap(f, d, mid) < 0.0)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* ELBM collision of one cell: f' = f + alpha beta (f_eq - f) + F_l with
 * beta = 1 / (2 tau0) (the effective relaxation time is tau_eff = 2 tau0 /
 * alpha, Sec. 1), f_eq the entropic equilibrium at u = j / rho, and the EDM
 * term F_l = f_eq(rho, u + F / rho) - f_eq(rho, u) with the same
 * equilibrium.  Returns alpha. */
double orc_elbm_cell(const double *fin, double tau0, double Fex, double Fey,
                     double alpha_drag, double *fout) {
  double rho, jx, jy;
  cell_moments(fin, &rho, &jx, &jy);
  double ux = jx / rho, uy = jy / rho;
  double Fx = Fex - alpha_drag * jx, Fy = Fey - alpha_drag * jy;
  double feq[Q], fsh[Q], d[Q];
  orc_feq_entropic(rho, ux, uy, feq);
  orc_feq_entropic(rho, ux + Fx / rho, uy + Fy / rho, fsh);
  for (int l = 0; l < Q; ++l) d[l] = feq[l] - fin[l];
  double a = orc_elbm_alpha(fin, d);
  double beta = 1.0 / (2.0 * tau0);
  for (int l = 0; l < Q; ++l) fout[l] = fin[l] + a * beta * d[l] + (fsh[l] - feq[l]);
  return a;
}

/* Local relaxation time of one cell (populations fc) for the member's
 * collision model.  The strain rate comes from the non-equilibrium second
 * moment of the pre-collision populations, Pi^neq = sum_l c c (f - f_eq),
 * f_eq = eq. (2) at u = j / rho, through the Chapman-Enskog relation
 * Pi^neq = -2 rho cs^2 tau S (S_ij = (d_i u_j + d_j u_i) / 2, dt = 1):
 *   Smagorinsky: tau = tau0 + nu_t / cs^2, nu_t = C sqrt(S:S), with S taken
 *     at tau itself: tau (tau - tau0) = C sqrt(Pi:Pi) / (2 rho cs^4), the
 *     positive root tau = (tau0 + sqrt(tau0^2 + 2 C |Pi| / (rho cs^4))) / 2;
 *   eq. (7): nu_t = -(cs^2 / 3) tau0^2 Tr(S^3) / Tr(S^2) with S taken at tau0
 *     (the formula assumes tau_eff ~ tau0), i.e. tau = tau0 + tau0 Tr(Pi^3)
 *     / (2 rho Tr(Pi^2)) (tau0 where Pi = 0). */
double orc_tau_eff(const double *fc, double tau0, const orc_model_t *P) {
  if (P->collision == 0) return tau0;
  if (P->collision == 3) { /* ELBM: tau_eff = 2 tau0 / alpha */
    double rho, jx, jy, feq[Q], d[Q];
    cell_moments(fc, &rho, &jx, &jy);
    orc_feq_entropic(rho, jx / rho, jy / rho, feq);
    for (int l = 0; l < Q; ++l) d[l] = feq[l] - fc[l];
    return 2.0 * tau0 / orc_elbm_alpha(fc, d);
  }
  double rho, jx, jy, feq[Q];
  cell_moments(fc, &rho, &jx, &jy);
  orc_feq(rho, jx / rho, jy / rho, feq);
  double pxx = 0.0, pxy = 0.0, pyy = 0.0;
  for (int l = 0; l < Q; ++l) {
    double d = fc[l] - feq[l];
    pxx += CX[l] * CX[l] * d;
    pxy += CX[l] * CY[l] * d;
    pyy += CY[l] * CY[l] * d;
  }
  double tr2 = pxx * pxx + 2.0 * pxy * pxy + pyy * pyy; /* Tr(Pi^2) = Pi:Pi */
  if (P->collision == 1) {
    double cs4 = CS2 * CS2;
    return 0.5 * (tau0 + sqrt(tau0 * tau0 + 2.0 * P->Cs * sqrt(tr2) / (rho * cs4)));
  }
  if (tr2 == 0.0) return tau0;
  /* Tr(Pi^3) of the symmetric 2 x 2 tensor, by matrix products */
  double a2xx = pxx * pxx + pxy * pxy, a2xy = pxx * pxy + pxy * pyy,
         a2yy = pxy * pxy + pyy * pyy;
  double tr3 = a2xx * pxx + 2.0 * a2xy * pxy + a2yy * pyy;
  return tau0 + tau0 * tr3 / (2.0 * rho * tr2);
}

/* Local viscosity of every cell of the state f, eq. (5) with the local
 * relaxation time: nu = cs^2 (tau_eff - 1/2). */
void orc_nu_field(int nx, int ny, double tau, const orc_model_t *P, const double *f,
                  double *nu) {
  size_t plane = (size_t)nx * ny;
  for (size_t c = 0; c < plane; ++c) {
    double a[Q];
    for (int l = 0; l < Q; ++l) a[l] = f[l * plane + c];
    nu[c] = CS2 * (orc_tau_eff(a, tau, P) - 0.5);
  }
}

/* Collision of the whole grid (no streaming): fout = fin + Omega(fin) + F,
 * with the external force of the state fin (orc_force_field). */
int orc_collide(int nx, int ny, double tau, const orc_model_t *F,
                const double *fin, double *fout) {
  size_t plane = (size_t)nx * ny;
  double *Fe = (double *)malloc(sizeof(double) * 2 * plane);
  if (!Fe) return -1;
  orc_force_field(nx, ny, F, fin, Fe, Fe + plane);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      double a[Q], b[Q];
      for (int l = 0; l < Q; ++l) a[l] = fin[l * plane + c];
      if (F->collision == 3)
        orc_elbm_cell(a, tau, Fe[c], Fe[plane + c], F->alpha, b);
      else
        orc_collide_cell(a, orc_tau_eff(a, tau, F), Fe[c], Fe[plane + c], F->alpha, b);
      for (int l = 0; l < Q; ++l) fout[l * plane + c] = b[l];
    }
  free(Fe);
  return 0;
}

/* Streaming, the left-hand side of eq. (1): f_l(x + c_l, n + 1) = f*_l(x),
 * periodic in both directions. */
void orc_stream(int nx, int ny, const double *fin, double *fout) {
  size_t plane = (size_t)nx * ny;
  for (int l = 0; l < Q; ++l)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int xd = wrap(x + CX[l], nx), yd = wrap(y + CY[l], ny);
        fout[l * plane + (size_t)yd * nx + xd] =
            fin[l * plane + (size_t)y * nx + x];
      }
}

/* One full time step of eq. (1): collide, then stream.  scratch holds one
 * population array (9 nx ny doubles).  f is updated in place. */
int orc_step(int nx, int ny, double tau, const orc_model_t *F, double *f,
             double *scratch) {
  if (orc_collide(nx, ny, tau, F, f, scratch)) return -1;
  orc_stream(nx, ny, scratch, f);
  return 0;
}

/* nsteps time steps; allocates its own scratch. */
int orc_run(int nx, int ny, double tau, const orc_model_t *F, double *f,
            int nsteps) {
  double *s = (double *)malloc(sizeof(double) * Q * (size_t)nx * ny);
  if (!s) return -1;
  int rc = 0;
  for (int n = 0; n < nsteps && rc == 0; ++n) rc = orc_step(nx, ny, tau, F, f, s);
  free(s);
  return rc;
}

/* nsteps time steps on a wx x wy window cut out of a larger NX x NY periodic
 * grid at global offset (X0, Y0): the same collide-then-stream as orc_step,
 * with the external force taken at the global coordinates
 * ((X0 + i) mod NX, (Y0 + j) mod NY) and the window treated as periodic.  A
 * step moves information by at most one cell, so after nsteps steps the
 * window cells at least nsteps cells away from its edges hold exactly the
 * values of the global run; the others are meaningless.  The damping of
 * kind 2 depends on the whole grid, so kind 2 is refused (-2). */
int orc_run_window(int wx, int wy, double tau, const orc_model_t *F, double *f,
                   int nsteps, int X0, int Y0, int NX, int NY) {
  if (F->kind == 2) return -2;
  size_t plane = (size_t)wx * wy;
  double *s = (double *)malloc(sizeof(double) * Q * plane);
  if (!s) return -1;
  for (int n = 0; n < nsteps; ++n) {
    for (int y = 0; y < wy; ++y)
      for (int x = 0; x < wx; ++x) {
        double a[Q], b[Q], Fex, Fey;
        for (int l = 0; l < Q; ++l) a[l] = f[l * plane + (size_t)y * wx + x];
        orc_force_ext(NX, NY, F, wrap(X0 + x, NX), wrap(Y0 + y, NY), &Fex, &Fey);
        if (F->collision == 3)
          orc_elbm_cell(a, tau, Fex, Fey, F->alpha, b);
        else
          orc_collide_cell(a, orc_tau_eff(a, tau, F), Fex, Fey, F->alpha, b);
        for (int l = 0; l < Q; ++l) s[l * plane + (size_t)y * wx + x] = b[l];
      }
    orc_stream(wx, wy, s, f);
  }
  free(s);
  return 0;
}

/* Initial state: f_l(x, 0) = f_eq_l(rho(x), u(x)). */
void orc_init(int nx, int ny, const double *rho, const double *ux,
              const double *uy, double *f) {
  size_t plane = (size_t)nx * ny;
  for (size_t c = 0; c < plane; ++c) {
    double e[Q];
    orc_feq(rho[c], ux[c], uy[c], e);
    for (int l = 0; l < Q; ++l) f[l * plane + c] = e[l];
  }
}

/* Moments of the state f(., n): rho, bare momentum j, and the EDM velocity
 * u_phys = (j + F/2)/rho with F = F_ext - alpha j.  Any output may be NULL. */
int orc_moments(int nx, int ny, const orc_model_t *F, const double *f,
                double *rho, double *jx, double *jy, double *ux, double *uy) {
  size_t plane = (size_t)nx * ny;
  double *Fe = (double *)malloc(sizeof(double) * 2 * plane);
  if (!Fe) return -1;
  orc_force_field(nx, ny, F, f, Fe, Fe + plane);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      double a[Q], r, px, py;
      for (int l = 0; l < Q; ++l) a[l] = f[l * plane + c];
      cell_moments(a, &r, &px, &py);
      double Fx = Fe[c] - F->alpha * px, Fy = Fe[plane + c] - F->alpha * py;
      if (rho) rho[c] = r;
      if (jx) jx[c] = px;
      if (jy) jy[c] = py;
      if (ux) ux[c] = (px + 0.5 * Fx) / r;
      if (uy) uy[c] = (py + 0.5 * Fy) / r;
    }
  free(Fe);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Finite differences, eqs. (17) and (18)                                   */
/* ------------------------------------------------------------------------ */

/* Eq. (18), x direction (first index), periodic, dx = 1:
 * (-A_{i+4}/56 + 4A_{i+3}/21 - A_{i+2} + 4A_{i+1}
 *  - 4A_{i-1} + A_{i-2} - 4A_{i-3}/21 + A_{i-4}/56) / 5. */
void orc_ddx(int nx, int ny, const double *A, double *out) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const double *r = A + (size_t)y * nx;
#define AX(d) r[wrap(x + (d), nx)]
      double s = -AX(4) / 56.0 + 4.0 * AX(3) / 21.0 - AX(2) + 4.0 * AX(1) -
                 4.0 * AX(-1) + AX(-2) - 4.0 * AX(-3) / 21.0 + AX(-4) / 56.0;
#undef AX
      out[(size_t)y * nx + x] = s / 5.0;
    }
}

/* Eq. (18), y direction (second index). */
void orc_ddy(int nx, int ny, const double *A, double *out) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
#define AY(d) A[(size_t)wrap(y + (d), ny) * nx + x]
      double s = -AY(4) / 56.0 + 4.0 * AY(3) / 21.0 - AY(2) + 4.0 * AY(1) -
                 4.0 * AY(-1) + AY(-2) - 4.0 * AY(-3) / 21.0 + AY(-4) / 56.0;
#undef AY
      out[(size_t)y * nx + x] = s / 5.0;
    }
}

/* Eq. (17): (3 A^n - 4 A^{n-1} + A^{n-2}) / (2 dt), dt = 1. */
void orc_bdf2(size_t n, const double *An, const double *An1, const double *An2,
              double *out) {
  for (size_t i = 0; i < n; ++i)
    out[i] = (3.0 * An[i] - 4.0 * An1[i] + An2[i]) / 2.0;
}

/* ------------------------------------------------------------------------ */
/* Local balance terms, eqs. (8)-(11) in 2D                                 */
/* ------------------------------------------------------------------------ */

/* Term-field order of the output (NT = 13 planes of nx*ny doubles):
 *   0 LHS^E, 1..5 RHS^{E,1..5}, 6 LHS^Omega, 7..12 RHS^{Omega,1..6}.
 * Inputs: rho, ux, uy (the EDM velocity) at time levels n, n-1, n-2
 * (index 0, 1, 2 of the arrays of pointers), and the total force (Fx, Fy)
 * at time n.  nu = cs^2 (tau - 1/2), eq. (5).  In 2D the vorticity is the
 * scalar w = d_x u_y - d_y u_x; the epsilon contractions of eqs. (9), (11)
 * reduce to
 *   H_i grad-cross:  H_x d_y w - H_y d_x w
 *   curl of F/rho:   d_x(F_y/rho) - d_y(F_x/rho)
 *   flux of w x H:   d_x(w H_y) - d_y(w H_x)
 *   stretching:      0.
 * The compressibility term of enstrophy follows eq. (11): -(w^2/2) div u. */
int orc_terms(int nx, int ny, double tau, const double *const *rho,
              const double *const *ux, const double *const *uy,
              const double *Fx, const double *Fy, const double *nu_field,
              double *terms) {
  size_t N = (size_t)nx * ny;
  const double nu0 = CS2 * (tau - 0.5);
#define NU(i) (nu_field ? nu_field[i] : nu0)
  /* scratch fields */
  enum {
    DXUX, DYUX, DXUY, DYUY, W0, W1, W2, E0, E1, E2, OM0, OM1, OM2,
    SXX, SXY, SYY, P, DXP, DYP, TMPA, TMPB, TMPC, TMPD, HX, HY, DXW, DYW,
    NSCR
  };
  double *s = (double *)malloc(sizeof(double) * N * NSCR);
  if (!s) return -1;
#define F_(k) (s + (size_t)(k) * N)
  double *T = terms;
#define T_(k) (T + (size_t)(k) * N)

  /* vorticity and energy at the three time levels */
  for (int m = 0; m < 3; ++m) {
    orc_ddx(nx, ny, uy[m], F_(TMPA));
    orc_ddy(nx, ny, ux[m], F_(TMPB));
    for (size_t i = 0; i < N; ++i) {
      double w = F_(TMPA)[i] - F_(TMPB)[i];
      F_(W0 + m)[i] = w;
      F_(OM0 + m)[i] = 0.5 * w * w;
      F_(E0 + m)[i] =
          0.5 * rho[m][i] * (ux[m][i] * ux[m][i] + uy[m][i] * uy[m][i]);
    }
  }
  /* LHS terms, eq. (17) */
  orc_bdf2(N, F_(E0), F_(E1), F_(E2), T_(0));
  orc_bdf2(N, F_(OM0), F_(OM1), F_(OM2), T_(6));

  const double *r = rho[0], *u = ux[0], *v = uy[0], *w = F_(W0),
               *Om = F_(OM0), *E = F_(E0);
  /* velocity gradients at time n */
  orc_ddx(nx, ny, u, F_(DXUX));
  orc_ddy(nx, ny, u, F_(DYUX));
  orc_ddx(nx, ny, v, F_(DXUY));
  orc_ddy(nx, ny, v, F_(DYUY));
  /* S_ij = d_j u_i + d_i u_j */
  for (size_t i = 0; i < N; ++i) {
    F_(SXX)[i] = 2.0 * F_(DXUX)[i];
    F_(SXY)[i] = F_(DYUX)[i] + F_(DXUY)[i];
    F_(SYY)[i] = 2.0 * F_(DYUY)[i];
    F_(P)[i] = CS2 * r[i]; /* p = cs^2 rho */
  }

  /* RHS^{E,1} = -d_j (E u_j) */
  for (size_t i = 0; i < N; ++i) {
    F_(TMPA)[i] = E[i] * u[i];
    F_(TMPB)[i] = E[i] * v[i];
  }
  orc_ddx(nx, ny, F_(TMPA), F_(TMPC));
  orc_ddy(nx, ny, F_(TMPB), F_(TMPD));
  for (size_t i = 0; i < N; ++i) T_(1)[i] = -(F_(TMPC)[i] + F_(TMPD)[i]);

  /* RHS^{E,2} = -u_i d_i p */
  orc_ddx(nx, ny, F_(P), F_(DXP));
  orc_ddy(nx, ny, F_(P), F_(DYP));
  for (size_t i = 0; i < N; ++i)
    T_(2)[i] = -(u[i] * F_(DXP)[i] + v[i] * F_(DYP)[i]);

  /* RHS^{E,3} = u_i F_i */
  for (size_t i = 0; i < N; ++i) T_(3)[i] = u[i] * Fx[i] + v[i] * Fy[i];

  /* RHS^{E,4} = -nu rho S_ij d_j u_i */
  for (size_t i = 0; i < N; ++i) {
    double sdu = F_(SXX)[i] * F_(DXUX)[i]   /* i=x, j=x */
                 + F_(SXY)[i] * F_(DYUX)[i] /* i=x, j=y: S_xy d_y u_x */
                 + F_(SXY)[i] * F_(DXUY)[i] /* i=y, j=x: S_yx d_x u_y */
                 + F_(SYY)[i] * F_(DYUY)[i];
    T_(4)[i] = -NU(i) * r[i] * sdu;
  }

  /* RHS^{E,5} = d_j (nu rho u_i S_ij) */
  for (size_t i = 0; i < N; ++i) {
    F_(TMPA)[i] = NU(i) * r[i] * (u[i] * F_(SXX)[i] + v[i] * F_(SXY)[i]); /* j=x */
    F_(TMPB)[i] = NU(i) * r[i] * (u[i] * F_(SXY)[i] + v[i] * F_(SYY)[i]); /* j=y */
  }
  orc_ddx(nx, ny, F_(TMPA), F_(TMPC));
  orc_ddy(nx, ny, F_(TMPB), F_(TMPD));
  for (size_t i = 0; i < N; ++i) T_(5)[i] = F_(TMPC)[i] + F_(TMPD)[i];

  /* H_i = (1/rho) d_j (nu rho S_ij) */
  for (size_t i = 0; i < N; ++i) {
    F_(TMPA)[i] = NU(i) * r[i] * F_(SXX)[i];
    F_(TMPB)[i] = NU(i) * r[i] * F_(SXY)[i];
  }
  orc_ddx(nx, ny, F_(TMPA), F_(TMPC));
  orc_ddy(nx, ny, F_(TMPB), F_(TMPD));
  for (size_t i = 0; i < N; ++i) F_(HX)[i] = (F_(TMPC)[i] + F_(TMPD)[i]) / r[i];
  for (size_t i = 0; i < N; ++i) {
    F_(TMPA)[i] = NU(i) * r[i] * F_(SXY)[i];
    F_(TMPB)[i] = NU(i) * r[i] * F_(SYY)[i];
  }
  orc_ddx(nx, ny, F_(TMPA), F_(TMPC));
  orc_ddy(nx, ny, F_(TMPB), F_(TMPD));
  for (size_t i = 0; i < N; ++i) F_(HY)[i] = (F_(TMPC)[i] + F_(TMPD)[i]) / r[i];

  /* RHS^{Omega,1} = -d_j (Omega u_j) */
  for (size_t i = 0; i < N; ++i) {
    F_(TMPA)[i] = Om[i] * u[i];
    F_(TMPB)[i] = Om[i] * v[i];
  }
  orc_ddx(nx, ny, F_(TMPA), F_(TMPC));
  orc_ddy(nx, ny, F_(TMPB), F_(TMPD));
  for (size_t i = 0; i < N; ++i) T_(7)[i] = -(F_(TMPC)[i] + F_(TMPD)[i]);

  /* RHS^{Omega,2} = -Omega d_j u_j */
  for (size_t i = 0; i < N; ++i)
    T_(8)[i] = -Om[i] * (F_(DXUX)[i] + F_(DYUY)[i]);

  /* RHS^{Omega,3} = w (d_x (F_y/rho) - d_y (F_x/rho)) */
  for (size_t i = 0; i < N; ++i) {
    F_(TMPA)[i] = Fy[i] / r[i];
    F_(TMPB)[i] = Fx[i] / r[i];
  }
  orc_ddx(nx, ny, F_(TMPA), F_(TMPC));
  orc_ddy(nx, ny, F_(TMPB), F_(TMPD));
  for (size_t i = 0; i < N; ++i) T_(9)[i] = w[i] * (F_(TMPC)[i] - F_(TMPD)[i]);

  /* RHS^{Omega,4} = H_x d_y w - H_y d_x w */
  orc_ddx(nx, ny, w, F_(DXW));
  orc_ddy(nx, ny, w, F_(DYW));
  for (size_t i = 0; i < N; ++i)
    T_(10)[i] = F_(HX)[i] * F_(DYW)[i] - F_(HY)[i] * F_(DXW)[i];

  /* RHS^{Omega,5} = d_x (w H_y) - d_y (w H_x) */
  for (size_t i = 0; i < N; ++i) {
    F_(TMPA)[i] = w[i] * F_(HY)[i];
    F_(TMPB)[i] = w[i] * F_(HX)[i];
  }
  orc_ddx(nx, ny, F_(TMPA), F_(TMPC));
  orc_ddy(nx, ny, F_(TMPB), F_(TMPD));
  for (size_t i = 0; i < N; ++i) T_(11)[i] = F_(TMPC)[i] - F_(TMPD)[i];

  /* RHS^{Omega,6} = w_i w_j d_j u_i = 0 in 2D (no vortex stretching) */
  for (size_t i = 0; i < N; ++i) T_(12)[i] = 0.0;

#undef F_
#undef T_
#undef NU
  free(s);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sub-volume averages and balancing errors, eqs. (10)-(13), Table 1        */
/* ------------------------------------------------------------------------ */

/* Average of field A over the L x L box with lower-left corner (x0, y0),
 * wrapping periodically: the <.>_V of eqs. (10), (11).  Brute force. */
double orc_box_mean(int nx, int ny, const double *A, int x0, int y0, int L) {
  double s = 0.0;
  for (int dy = 0; dy < L; ++dy)
    for (int dx = 0; dx < L; ++dx)
      s += A[(size_t)wrap(y0 + dy, ny) * nx + wrap(x0 + dx, nx)];
  return s / ((double)L * (double)L);
}

/* Balancing errors of eqs. (12), (13) for one box, from the 13 box-averaged
 * terms (order as in orc_terms).  A zero denominator gives 0 when the
 * numerator is 0 and +Inf otherwise. */
static double delta_of(const double *lhs_rhs, int nrhs) {
  double lhs = lhs_rhs[0], sum = 0.0, mx = 0.0;
  for (int i = 1; i <= nrhs; ++i) {
    sum += lhs_rhs[i];
    if (fabs(lhs_rhs[i]) > mx) mx = fabs(lhs_rhs[i]);
  }
  double num = fabs(sum - lhs);
  if (mx == 0.0) return num == 0.0 ? 0.0 : INFINITY;
  return num / mx;
}

void orc_box_values(int nx, int ny, const double *terms, int x0, int y0, int L,
                    double *out15) {
  size_t N = (size_t)nx * ny;
  double b[13];
  for (int k = 0; k < 13; ++k)
    b[k] = orc_box_mean(nx, ny, terms + (size_t)k * N, x0, y0, L);
  out15[0] = delta_of(b, 5);     /* delta^E: LHS^E, RHS^{E,1..5} */
  out15[1] = delta_of(b + 6, 6); /* delta^Omega: LHS^O, RHS^{O,1..6} */
  for (int k = 0; k < 13; ++k) out15[2 + k] = b[k];
}

/* Statistics over boxes of each size L (Sec. 3: mean mu_l and standard deviation
 * sigma_l of Sec. 3), for the 15 box quantities
 *   [delta^E, delta^Omega, LHS^E, RHS^{E,1..5}, LHS^O, RHS^{O,1..6}].
 * Boxes: all nx*ny periodic origins when origins == NULL, else the
 * n_origins (x0, y0) pairs of origins[2*i], origins[2*i+1] (used for every
 * L).  Sizes L > min(nx, ny) are skipped (their statistics are NaN).
 * stats[(iL*15 + q)*2 + 0] = mean, [...+1] = population standard deviation.
 * per_box, if not NULL, receives [iL][box][15]. */
int orc_balance_stats(int nx, int ny, const double *terms, const int *Ls,
                      int nL, const int *origins, int n_origins, double *stats,
                      double *per_box) {
  int nb = origins ? n_origins : nx * ny;
  double *vals = (double *)malloc(sizeof(double) * 15 * (size_t)nb);
  if (!vals) return -1;
  for (int iL = 0; iL < nL; ++iL) {
    int L = Ls[iL];
    double *st = stats + (size_t)iL * 30;
    if (L < 1 || L > nx || L > ny) {
      for (int q = 0; q < 30; ++q) st[q] = NAN;
      continue;
    }
    for (int b = 0; b < nb; ++b) {
      int x0 = origins ? origins[2 * b] : b % nx;
      int y0 = origins ? origins[2 * b + 1] : b / nx;
      orc_box_values(nx, ny, terms, x0, y0, L, vals + (size_t)b * 15);
    }
    for (int q = 0; q < 15; ++q) {
      double m = 0.0;
      for (int b = 0; b < nb; ++b) m += vals[(size_t)b * 15 + q];
      m /= nb;
      double v = 0.0;
      for (int b = 0; b < nb; ++b) {
        double d = vals[(size_t)b * 15 + q] - m;
        v += d * d;
      }
      st[2 * q] = m;
      st[2 * q + 1] = sqrt(v / nb);
    }
    if (per_box)
      memcpy(per_box + (size_t)iL * nb * 15, vals, sizeof(double) * 15 * nb);
  }
  free(vals);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Distributions over boxes: sub-volume Mach number (eq. 20), PDFs (Sec. 4) */
/* ------------------------------------------------------------------------ */

/* Sub-volume Mach number of eq. (20), read as the RMS speed over the L x L
 * box (lower-left origin (x0, y0), periodic) divided by the lattice speed of
 * sound: Ma_V = sqrt(<u_x^2 + u_y^2>_V) / c_s, u the diagnostic velocity. */
double orc_box_mach(int nx, int ny, const double *ux, const double *uy, int x0,
                    int y0, int L) {
  double s = 0.0;
  for (int dy = 0; dy < L; ++dy)
    for (int dx = 0; dx < L; ++dx) {
      size_t c = (size_t)wrap(y0 + dy, ny) * nx + wrap(x0 + dx, nx);
      s += ux[c] * ux[c] + uy[c] * uy[c];
    }
  return sqrt(s / ((double)L * (double)L)) / sqrt(CS2);
}

/* Histogram bin of v for ascending edges e[0..n-1]: the number of edges
 * e_k <= v, so bin 0 holds v < e_0, bin k holds e_{k-1} <= v < e_k and bin n
 * holds v >= e_{n-1} (+Inf included).  NaN belongs to no bin (-1). */
int orc_bin(double v, const double *edges, int n) {
  if (v != v) return -1;
  int b = 0;
  while (b < n && edges[b] <= v) ++b;
  return b;
}

/* Distributions over the boxes of each size: the histograms behind the PDFs
 * of the balancing errors shown in Sec. 4 and the mean and standard
 * deviation of Ma_V (eq. 20) shown there against l.
 *   hist_delta[(iL*2 + q)*(n_de + 1) + b]: boxes whose delta^E (q = 0) or
 *     delta^Omega (q = 1) lies in bin b of delta_edges;
 *   hist_mach[iL*(n_me + 1) + b]: the same for Ma_V and mach_edges;
 *   mach_stats[iL*2 + 0 / 1]: mean and population standard deviation of Ma_V.
 * Boxes as in orc_balance_stats; a size L > min(nx, ny) gives zero counts
 * and NaN statistics. */
int orc_distributions(int nx, int ny, const double *terms, const double *ux,
                      const double *uy, const int *Ls, int nL,
                      const int *origins, int n_origins,
                      const double *delta_edges, int n_de,
                      const double *mach_edges, int n_me,
                      long long *hist_delta, long long *hist_mach,
                      double *mach_stats) {
  int nb = origins ? n_origins : nx * ny;
  double *ma = (double *)malloc(sizeof(double) * (size_t)nb);
  if (!ma) return -1;
  for (int iL = 0; iL < nL; ++iL) {
    int L = Ls[iL];
    long long *hd = hist_delta + (size_t)iL * 2 * (n_de + 1);
    long long *hm = hist_mach + (size_t)iL * (n_me + 1);
    for (int b = 0; b < 2 * (n_de + 1); ++b) hd[b] = 0;
    for (int b = 0; b <= n_me; ++b) hm[b] = 0;
    if (L < 1 || L > nx || L > ny) {
      mach_stats[2 * iL] = NAN;
      mach_stats[2 * iL + 1] = NAN;
      continue;
    }
    for (int b = 0; b < nb; ++b) {
      int x0 = origins ? origins[2 * b] : b % nx;
      int y0 = origins ? origins[2 * b + 1] : b / nx;
      double v[15];
      orc_box_values(nx, ny, terms, x0, y0, L, v);
      for (int q = 0; q < 2; ++q) {
        int k = orc_bin(v[q], delta_edges, n_de);
        if (k >= 0) hd[q * (n_de + 1) + k] += 1;
      }
      ma[b] = orc_box_mach(nx, ny, ux, uy, x0, y0, L);
      int k = orc_bin(ma[b], mach_edges, n_me);
      if (k >= 0) hm[k] += 1;
    }
    double m = 0.0, var = 0.0;
    for (int b = 0; b < nb; ++b) m += ma[b];
    m /= nb;
    for (int b = 0; b < nb; ++b) var += (ma[b] - m) * (ma[b] - m);
    mach_stats[2 * iL] = m;
    mach_stats[2 * iL + 1] = sqrt(var / nb);
  }
  free(ma);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Convenience: diagnostic from three population snapshots                  */
/* ------------------------------------------------------------------------ */

/* Term fields at time n from the pre-collision populations at n, n-1, n-2
 * (f_n, f_n1, f_n2), using u_phys and F = F_ext - alpha j at each level and,
 * for a variable-viscosity collision, the local viscosity of the state at
 * time n. */
int orc_terms_from_populations(int nx, int ny, double tau, const orc_model_t *F,
                               const double *f_n, const double *f_n1,
                               const double *f_n2, double *terms) {
  size_t N = (size_t)nx * ny;
  double *buf = (double *)malloc(sizeof(double) * N * 13);
  if (!buf) return -1;
  double *rho[3], *ux[3], *uy[3], *jx = buf + 9 * N, *jy = buf + 10 * N,
                                  *Fx = buf + 11 * N, *Fy = buf + 12 * N;
  const double *fs[3] = {f_n, f_n1, f_n2};
  for (int m = 0; m < 3; ++m) {
    rho[m] = buf + (3 * m + 0) * N;
    ux[m] = buf + (3 * m + 1) * N;
    uy[m] = buf + (3 * m + 2) * N;
    if (orc_moments(nx, ny, F, fs[m], rho[m], jx, jy, ux[m], uy[m])) {
      free(buf);
      return -1;
    }
    if (m == 0) {
      orc_force_field(nx, ny, F, fs[0], Fx, Fy);
      for (size_t c = 0; c < N; ++c) {
        Fx[c] -= F->alpha * jx[c];
        Fy[c] -= F->alpha * jy[c];
      }
    }
  }
  double *nu = NULL;
  if (F->collision != 0) {
    nu = (double *)malloc(sizeof(double) * N);
    if (!nu) {
      free(buf);
      return -1;
    }
    orc_nu_field(nx, ny, tau, F, f_n, nu);
  }
  int rc = orc_terms(nx, ny, tau, (const double *const *)rho,
                     (const double *const *)ux, (const double *const *)uy, Fx,
                     Fy, nu, terms);
  free(nu);
  free(buf);
  return rc;
}

/* Whole-grid quantities of the state f(., n), all FP64:
 *   out[0] = sum rho, out[1] = sum j_x, out[2] = sum j_y,
 *   out[3] = <E> = mean rho |u|^2 / 2,  out[4] = <Omega> = mean w^2 / 2,
 *   out[5] = <u . F>,  out[6] = <eps> = mean nu rho S_ij d_j u_i
 * with u = u_phys and the eq. (18) derivatives. */
int orc_global(int nx, int ny, double tau, const orc_model_t *F,
               const double *f, double *out) {
  size_t N = (size_t)nx * ny;
  double *b = (double *)malloc(sizeof(double) * N * 11);
  if (!b) return -1;
  double *rho = b, *jx = b + N, *jy = b + 2 * N, *u = b + 3 * N,
         *v = b + 4 * N, *dxu = b + 5 * N, *dyu = b + 6 * N, *dxv = b + 7 * N,
         *dyv = b + 8 * N;
  double *Fe = (double *)malloc(sizeof(double) * N * 2);
  if (!Fe || orc_moments(nx, ny, F, f, rho, jx, jy, u, v)) {
    free(b);
    free(Fe);
    return -1;
  }
  orc_force_field(nx, ny, F, f, Fe, Fe + N);
  orc_ddx(nx, ny, u, dxu);
  orc_ddy(nx, ny, u, dyu);
  orc_ddx(nx, ny, v, dxv);
  orc_ddy(nx, ny, v, dyv);
  double *nu = b + 9 * N; /* local viscosity of the state */
  orc_nu_field(nx, ny, tau, F, f, nu);
  double s[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      double Fx = Fe[c] - F->alpha * jx[c], Fy = Fe[N + c] - F->alpha * jy[c];
      double w = dxv[c] - dyu[c];
      double sxx = 2 * dxu[c], sxy = dyu[c] + dxv[c], syy = 2 * dyv[c];
      s[0] += rho[c];
      s[1] += jx[c];
      s[2] += jy[c];
      s[3] += 0.5 * rho[c] * (u[c] * u[c] + v[c] * v[c]);
      s[4] += 0.5 * w * w;
      s[5] += u[c] * Fx + v[c] * Fy;
      s[6] += nu[c] * rho[c] *
              (sxx * dxu[c] + sxy * dyu[c] + sxy * dxv[c] + syy * dyv[c]);
    }
  out[0] = s[0];
  out[1] = s[1];
  out[2] = s[2];
  for (int k = 3; k < 7; ++k) out[k] = s[k] / (double)N;
  free(b);
  free(Fe);
  return 0;
}

/* Objective of the differentiation workload: J = (1/(n1-n0+1)) sum over
 * n in [n0, n1] of the L x L box average (origin (bx, by)) of RHS^{E,4}(n),
 * the local dissipation term of eq. (8), evaluated on the state f(., n).
 * Runs the forward model from f0 (copied, not modified) for n1 steps. */
int orc_objective(int nx, int ny, double tau, const orc_model_t *F,
                  const double *f0, int n0, int n1, int bx, int by, int L,
                  double *J) {
  size_t N = (size_t)nx * ny;
  double *f = (double *)malloc(sizeof(double) * Q * N);
  double *s = (double *)malloc(sizeof(double) * Q * N);
  double *b = (double *)malloc(sizeof(double) * N * 10);
  if (!f || !s || !b) {
    free(f);
    free(s);
    free(b);
    return -1;
  }
  memcpy(f, f0, sizeof(double) * Q * N);
  double *rho = b, *jx = b + N, *jy = b + 2 * N, *u = b + 3 * N,
         *v = b + 4 * N, *dxu = b + 5 * N, *dyu = b + 6 * N, *dxv = b + 7 * N,
         *dyv = b + 8 * N, *eps = b + 9 * N;
  double nu = CS2 * (tau - 0.5), acc = 0.0;
  for (int n = 0; n <= n1; ++n) {
    if (n >= n0) {
      orc_moments(nx, ny, F, f, rho, jx, jy, u, v);
      orc_ddx(nx, ny, u, dxu);
      orc_ddy(nx, ny, u, dyu);
      orc_ddx(nx, ny, v, dxv);
      orc_ddy(nx, ny, v, dyv);
      for (size_t c = 0; c < N; ++c) {
        double sxx = 2 * dxu[c], sxy = dyu[c] + dxv[c], syy = 2 * dyv[c];
        eps[c] = -nu * rho[c] *
                 (sxx * dxu[c] + sxy * dyu[c] + sxy * dxv[c] + syy * dyv[c]);
      }
      acc += orc_box_mean(nx, ny, eps, bx, by, L);
    }
    if (n < n1) orc_step(nx, ny, tau, F, f, s);
  }
  *J = acc / (double)(n1 - n0 + 1);
  free(f);
  free(s);
  free(b);
  return 0;
}
