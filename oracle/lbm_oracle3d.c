/*
 * Oracle for the three-dimensional extension of the method of Tauzin,
 * Biferale, Sbragaglia, Gupta, Toschi, Bartel, Ehrhardt (Comput. & Fluids
 * 172, 2018): the D3Q19 and D3Q27 lattice BGK of eq. (1) with the eq. (2) equilibrium
 * and exact-difference forcing, and the sub-volume energy and enstrophy
 * balance of eqs. (8)-(13) in their general index forms, where the vortex
 * stretching term RHS^{Omega,6} = omega_i omega_j d_j u_i no longer vanishes
 * (the paper's outlook names D3Q19/D3Q27 with vortex stretching).
 *
 * TEST INFRASTRUCTURE ONLY, like lbm_oracle.c: plain, slow, FP64, single
 * threaded; it shares nothing with the CUDA library and only the test-suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Conventions (readings listed in the design notes of the repository):
 *   - D3Q19 order: c_0 = 0; c_1..6 = +x, -x, +y, -y, +z, -z;
 *     c_7..18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1),
 *     (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1);
 *     weights 1/3, 1/18, 1/36; c_s^2 = 1/3.
 *   - D3Q27 order: the D3Q19 order, then the corners c_19..26 = (1,1,1),
 *     (-1,-1,-1), (1,1,-1), (-1,-1,1), (1,-1,1), (-1,1,-1), (-1,1,1),
 *     (1,-1,-1); weights 8/27, 2/27, 1/54, 1/216 by |c|^2 = 0..3.  The
 *     lattice is the first argument (q = 19 or 27) of every function that
 *     touches populations.
 *   - Arrays: f[((l nz + z) ny + y) nx + x], fields A[(z ny + y) nx + x].
 *   - Force kind 1: F_ext = F0 (sin(2 pi kf y/ny), sin(2 pi kf z/nz),
 *     sin(2 pi kf x/nx)), plus drag -alpha j; EDM as in two dimensions.
 *   - Diagnostic velocity u = (j + F/2)/rho; boxes L x L x L with lower
 *     corner (x0, y0, z0), wrapping periodically.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Velocity sets.  D3Q27 = rest, 6 axis, 12 edge and 8 corner velocities;
 * D3Q19 is its first 19 entries (no corners).  Weights by |c|^2:
 *   D3Q19: 1/3, 1/18, 1/36;  D3Q27: 8/27, 2/27, 1/54, 1/216;
 * both with c_s^2 = 1/3 and the same eq. (2) equilibrium. */
#define QMAX 27
static const int C3X[QMAX] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0,
                              1, -1, 1, -1, 1, -1, -1, 1};
static const int C3Y[QMAX] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1,
                              1, -1, 1, -1, -1, 1, 1, -1};
static const int C3Z[QMAX] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1,
                              1, -1, -1, 1, 1, -1, 1, -1};
static const double CS2_3 = 1.0 / 3.0;
static const double PI3 = 3.14159265358979323846;

static double w3(int q, int l) {
  const int c2 = C3X[l] * C3X[l] + C3Y[l] * C3Y[l] + C3Z[l] * C3Z[l];
  if (q == 27) return c2 == 0 ? 8.0 / 27.0 : (c2 == 1 ? 2.0 / 27.0 : (c2 == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
  return c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

static int valid_q(int q) { return q == 19 || q == 27; }

static int wrap3(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

/* The lattice of q = 19 or 27 velocities; returns -1 for another q. */
int orc3_lattice(int q, int *cx, int *cy, int *cz, double *t) {
  if (!valid_q(q)) return -1;
  for (int l = 0; l < q; ++l) {
    cx[l] = C3X[l];
    cy[l] = C3Y[l];
    cz[l] = C3Z[l];
    t[l] = w3(q, l);
  }
  return 0;
}

/* Eq. (2) on D3Qq. */
void orc3_feq(int q, double rho, double ux, double uy, double uz, double *feq) {
  double uu = ux * ux + uy * uy + uz * uz;
  for (int l = 0; l < q; ++l) {
    double cu = C3X[l] * ux + C3Y[l] * uy + C3Z[l] * uz;
    feq[l] = w3(q, l) * rho * (1.0 + cu / CS2_3 + cu * cu / (2.0 * CS2_3 * CS2_3) - uu / (2.0 * CS2_3));
  }
}

void orc3_force_ext(int nx, int ny, int nz, int kind, double F0, int kf, int x, int y,
                    int z, double *Fx, double *Fy, double *Fz) {
  if (kind == 1) {
    *Fx = F0 * sin(2.0 * PI3 * kf * (double)y / ny);
    *Fy = F0 * sin(2.0 * PI3 * kf * (double)z / nz);
    *Fz = F0 * sin(2.0 * PI3 * kf * (double)x / nx);
  } else {
    *Fx = *Fy = *Fz = 0.0;
  }
}

static void moments3(int q, const double *fc, double *rho, double *jx, double *jy, double *jz) {
  double r = 0, a = 0, b = 0, c = 0;
  for (int l = 0; l < q; ++l) {
    r += fc[l];
    a += C3X[l] * fc[l];
    b += C3Y[l] * fc[l];
    c += C3Z[l] * fc[l];
  }
  *rho = r;
  *jx = a;
  *jy = b;
  *jz = c;
}

/* BGK collision of one cell with the EDM term, F = F_ext - alpha j. */
void orc3_collide_cell(int q, const double *fin, double tau, double Fex, double Fey, double Fez,
                       double alpha, double *fout) {
  double rho, jx, jy, jz;
  moments3(q, fin, &rho, &jx, &jy, &jz);
  double ux = jx / rho, uy = jy / rho, uz = jz / rho;
  double Fx = Fex - alpha * jx, Fy = Fey - alpha * jy, Fz = Fez - alpha * jz;
  double feq[QMAX], fsh[QMAX];
  orc3_feq(q, rho, ux, uy, uz, feq);
  orc3_feq(q, rho, ux + Fx / rho, uy + Fy / rho, uz + Fz / rho, fsh);
  for (int l = 0; l < q; ++l) fout[l] = fin[l] - (fin[l] - feq[l]) / tau + (fsh[l] - feq[l]);
}

/* One step of eq. (1): collide, then stream f_l(x + c_l) = f*_l(x). */
int orc3_step(int q, int nx, int ny, int nz, double tau, int kind, double F0, int kf,
              double alpha, double *f, double *s) {
  if (!valid_q(q)) return -1;
  size_t N = (size_t)nx * ny * nz;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t c = ((size_t)z * ny + y) * nx + x;
        double a[QMAX], b[QMAX], Fx, Fy, Fz;
        for (int l = 0; l < q; ++l) a[l] = f[l * N + c];
        orc3_force_ext(nx, ny, nz, kind, F0, kf, x, y, z, &Fx, &Fy, &Fz);
        orc3_collide_cell(q, a, tau, Fx, Fy, Fz, alpha, b);
        for (int l = 0; l < q; ++l) {
          size_t d = ((size_t)wrap3(z + C3Z[l], nz) * ny + wrap3(y + C3Y[l], ny)) * nx +
                     wrap3(x + C3X[l], nx);
          s[l * N + d] = b[l];
        }
      }
  memcpy(f, s, sizeof(double) * q * N);
  return 0;
}

int orc3_run(int q, int nx, int ny, int nz, double tau, int kind, double F0, int kf,
             double alpha, double *f, int nsteps) {
  if (!valid_q(q)) return -1;
  double *s = (double *)malloc(sizeof(double) * q * (size_t)nx * ny * nz);
  if (!s) return -1;
  for (int n = 0; n < nsteps; ++n) orc3_step(q, nx, ny, nz, tau, kind, F0, kf, alpha, f, s);
  free(s);
  return 0;
}

void orc3_init(int q, int nx, int ny, int nz, const double *rho, const double *ux,
               const double *uy, const double *uz, double *f) {
  size_t N = (size_t)nx * ny * nz;
  for (size_t c = 0; c < N; ++c) {
    double e[QMAX];
    orc3_feq(q, rho[c], ux[c], uy[c], uz[c], e);
    for (int l = 0; l < q; ++l) f[l * N + c] = e[l];
  }
}

/* rho, bare momentum j and u = (j + F/2)/rho (F = F_ext - alpha j); any
 * output may be NULL. */
void orc3_moments(int q, int nx, int ny, int nz, int kind, double F0, int kf, double alpha,
                  const double *f, double *rho, double *ux, double *uy, double *uz,
                  double *Fx_out, double *Fy_out, double *Fz_out) {
  size_t N = (size_t)nx * ny * nz;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t c = ((size_t)z * ny + y) * nx + x;
        double a[QMAX], r, jx, jy, jz, Fex, Fey, Fez;
        for (int l = 0; l < q; ++l) a[l] = f[l * N + c];
        moments3(q, a, &r, &jx, &jy, &jz);
        orc3_force_ext(nx, ny, nz, kind, F0, kf, x, y, z, &Fex, &Fey, &Fez);
        double Fx = Fex - alpha * jx, Fy = Fey - alpha * jy, Fz = Fez - alpha * jz;
        if (rho) rho[c] = r;
        if (ux) ux[c] = (jx + 0.5 * Fx) / r;
        if (uy) uy[c] = (jy + 0.5 * Fy) / r;
        if (uz) uz[c] = (jz + 0.5 * Fz) / r;
        if (Fx_out) Fx_out[c] = Fx;
        if (Fy_out) Fy_out[c] = Fy;
        if (Fz_out) Fz_out[c] = Fz;
      }
}

/* Eq. (18) along axis `axis` (0 x, 1 y, 2 z), periodic, dx = 1. */
void orc3_d(int nx, int ny, int nz, int axis, const double *A, double *out) {
  static const double cf[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double s = 0.0;
        for (int k = 1; k <= 4; ++k) {
          int xp = x, xm = x, yp = y, ym = y, zp = z, zm = z;
          if (axis == 0) { xp = wrap3(x + k, nx); xm = wrap3(x - k, nx); }
          if (axis == 1) { yp = wrap3(y + k, ny); ym = wrap3(y - k, ny); }
          if (axis == 2) { zp = wrap3(z + k, nz); zm = wrap3(z - k, nz); }
          s += cf[k - 1] * (A[((size_t)zp * ny + yp) * nx + xp] - A[((size_t)zm * ny + ym) * nx + xm]);
        }
        out[((size_t)z * ny + y) * nx + x] = s;
      }
}

/* The 13 term fields of eqs. (10), (11) in three dimensions at time n from
 * (rho, u) at n, n-1, n-2 (index 0, 1, 2) and F at n, in the order
 * LHS^E, RHS^{E,1..5}, LHS^O, RHS^{O,1..6}:
 *   RHS^{E,1} = -d_j(E u_j), RHS^{E,2} = -u_i d_i p (p = rho/3),
 *   RHS^{E,3} = u_i F_i, RHS^{E,4} = -nu rho S_ij d_j u_i,
 *   RHS^{E,5} = d_j(nu rho u_i S_ij), S_ij = d_j u_i + d_i u_j;
 *   omega = curl u, Omega = omega.omega/2, H_i = d_j(nu rho S_ij)/rho,
 *   RHS^{O,1} = -d_j(Omega u_j), RHS^{O,2} = -Omega d_j u_j,
 *   RHS^{O,3} = omega . curl(F/rho), RHS^{O,4} = H . curl(omega),
 *   RHS^{O,5} = d_j(eps_ijk omega_i H_k) = div(H x omega),
 *   RHS^{O,6} = omega_i omega_j d_j u_i (vortex stretching);
 * eq. (18) in space, eq. (17) in time. */
int orc3_terms(int nx, int ny, int nz, double tau, const double *const *rho,
               const double *const *ux, const double *const *uy, const double *const *uz,
               const double *Fx, const double *Fy, const double *Fz, double *T) {
  size_t N = (size_t)nx * ny * nz;
  const double nu = CS2_3 * (tau - 0.5);
  /* scratch: gradients g[i][j] = d_j u_i at n (9), omega at 3 levels (9),
   * E (3), Om (3), S (9 incl. symmetric), H (3), curl omega (3), work (6) */
  double *b = (double *)malloc(sizeof(double) * N * 48);
  if (!b) return -1;
  double *G[3][3], *W[3][3], *Ev[3], *Ov[3], *H[3], *CW[3], *t0 = b + 42 * N, *t1 = b + 43 * N,
         *t2 = b + 44 * N, *t3 = b + 45 * N, *t4 = b + 46 * N;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      G[i][j] = b + (3 * i + j) * N;
      W[i][j] = b + (9 + 3 * i + j) * N; /* level i, component j */
    }
  for (int m = 0; m < 3; ++m) {
    Ev[m] = b + (18 + m) * N;
    Ov[m] = b + (21 + m) * N;
    H[m] = b + (24 + m) * N;
    CW[m] = b + (27 + m) * N;
  }
  double *Sij[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Sij[i][j] = b + (30 + 3 * i + j) * N;
  /* omega, E, Omega at the three levels */
  for (int m = 0; m < 3; ++m) {
    const double *U[3] = {ux[m], uy[m], uz[m]};
    double *D[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) D[i][j] = G[i][j]; /* reused per level */
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) orc3_d(nx, ny, nz, j, U[i], D[i][j]);
    for (size_t c = 0; c < N; ++c) {
      double wx = D[2][1][c] - D[1][2][c], wy = D[0][2][c] - D[2][0][c],
             wz = D[1][0][c] - D[0][1][c];
      W[m][0][c] = wx;
      W[m][1][c] = wy;
      W[m][2][c] = wz;
      Ov[m][c] = 0.5 * (wx * wx + wy * wy + wz * wz);
      Ev[m][c] = 0.5 * rho[m][c] * (U[0][c] * U[0][c] + U[1][c] * U[1][c] + U[2][c] * U[2][c]);
    }
  }
  /* gradients at level n (the last loop left level 2 in G) */
  const double *U0[3] = {ux[0], uy[0], uz[0]};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) orc3_d(nx, ny, nz, j, U0[i], G[i][j]);
  const double *r = rho[0];
  double *T_[13];
  for (int q = 0; q < 13; ++q) T_[q] = T + (size_t)q * N;
  /* eq. (17) */
  for (size_t c = 0; c < N; ++c) {
    T_[0][c] = 1.5 * Ev[0][c] - 2.0 * Ev[1][c] + 0.5 * Ev[2][c];
    T_[6][c] = 1.5 * Ov[0][c] - 2.0 * Ov[1][c] + 0.5 * Ov[2][c];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (size_t c = 0; c < N; ++c) Sij[i][j][c] = G[i][j][c] + G[j][i][c];
  /* RHS^{E,1} = -d_j (E u_j); RHS^{O,1} = -d_j (Omega u_j) */
  for (int which = 0; which < 2; ++which) {
    const double *A = which ? Ov[0] : Ev[0];
    double *out = which ? T_[7] : T_[1];
    for (size_t c = 0; c < N; ++c) out[c] = 0.0;
    for (int j = 0; j < 3; ++j) {
      for (size_t c = 0; c < N; ++c) t0[c] = A[c] * U0[j][c];
      orc3_d(nx, ny, nz, j, t0, t1);
      for (size_t c = 0; c < N; ++c) out[c] -= t1[c];
    }
  }
  /* RHS^{E,2} = -u_i d_i p */
  for (size_t c = 0; c < N; ++c) { t0[c] = CS2_3 * r[c]; T_[2][c] = 0.0; }
  for (int i = 0; i < 3; ++i) {
    orc3_d(nx, ny, nz, i, t0, t1);
    for (size_t c = 0; c < N; ++c) T_[2][c] -= U0[i][c] * t1[c];
  }
  /* RHS^{E,3} = u_i F_i, RHS^{E,4} = -nu rho S_ij d_j u_i, RHS^{O,2}, RHS^{O,6} */
  for (size_t c = 0; c < N; ++c) {
    T_[3][c] = U0[0][c] * Fx[c] + U0[1][c] * Fy[c] + U0[2][c] * Fz[c];
    double sd = 0.0, st = 0.0, div = G[0][0][c] + G[1][1][c] + G[2][2][c];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        sd += Sij[i][j][c] * G[i][j][c];
        st += W[0][i][c] * W[0][j][c] * G[i][j][c];
      }
    T_[4][c] = -nu * r[c] * sd;
    T_[8][c] = -Ov[0][c] * div;
    T_[12][c] = st;
  }
  /* RHS^{E,5} = d_j (nu rho u_i S_ij) */
  for (size_t c = 0; c < N; ++c) T_[5][c] = 0.0;
  for (int j = 0; j < 3; ++j) {
    for (size_t c = 0; c < N; ++c)
      t0[c] = nu * r[c] * (U0[0][c] * Sij[0][j][c] + U0[1][c] * Sij[1][j][c] + U0[2][c] * Sij[2][j][c]);
    orc3_d(nx, ny, nz, j, t0, t1);
    for (size_t c = 0; c < N; ++c) T_[5][c] += t1[c];
  }
  /* H_i = d_j (nu rho S_ij) / rho */
  for (int i = 0; i < 3; ++i) {
    for (size_t c = 0; c < N; ++c) H[i][c] = 0.0;
    for (int j = 0; j < 3; ++j) {
      for (size_t c = 0; c < N; ++c) t0[c] = nu * r[c] * Sij[i][j][c];
      orc3_d(nx, ny, nz, j, t0, t1);
      for (size_t c = 0; c < N; ++c) H[i][c] += t1[c];
    }
    for (size_t c = 0; c < N; ++c) H[i][c] /= r[c];
  }
  /* curl(F / rho) and RHS^{O,3} = omega . curl(F / rho) */
  {
    const double *F[3] = {Fx, Fy, Fz};
    double *Fr[3] = {t2, t3, t4};
    for (int k = 0; k < 3; ++k)
      for (size_t c = 0; c < N; ++c) Fr[k][c] = F[k][c] / r[c];
    for (size_t c = 0; c < N; ++c) T_[9][c] = 0.0;
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3, k = (i + 2) % 3; /* (curl A)_i = d_j A_k - d_k A_j */
      orc3_d(nx, ny, nz, j, Fr[k], t0);
      orc3_d(nx, ny, nz, k, Fr[j], t1);
      for (size_t c = 0; c < N; ++c) T_[9][c] += W[0][i][c] * (t0[c] - t1[c]);
    }
  }
  /* curl omega and RHS^{O,4} = H . curl(omega) */
  for (size_t c = 0; c < N; ++c) T_[10][c] = 0.0;
  for (int i = 0; i < 3; ++i) {
    int j = (i + 1) % 3, k = (i + 2) % 3;
    orc3_d(nx, ny, nz, j, W[0][k], t0);
    orc3_d(nx, ny, nz, k, W[0][j], t1);
    for (size_t c = 0; c < N; ++c) {
      CW[i][c] = t0[c] - t1[c];
      T_[10][c] += H[i][c] * CW[i][c];
    }
  }
  /* RHS^{O,5} = d_j (H x omega)_j */
  for (size_t c = 0; c < N; ++c) T_[11][c] = 0.0;
  for (int jj = 0; jj < 3; ++jj) {
    int a = (jj + 1) % 3, bb = (jj + 2) % 3; /* (H x w)_j = H_a w_b - H_b w_a */
    for (size_t c = 0; c < N; ++c) t0[c] = H[a][c] * W[0][bb][c] - H[bb][c] * W[0][a][c];
    orc3_d(nx, ny, nz, jj, t0, t1);
    for (size_t c = 0; c < N; ++c) T_[11][c] += t1[c];
  }
  free(b);
  return 0;
}

int orc3_terms_from_populations(int q, int nx, int ny, int nz, double tau, int kind, double F0,
                                int kf, double alpha, const double *f_n, const double *f_n1,
                                const double *f_n2, double *terms) {
  if (!valid_q(q)) return -1;
  size_t N = (size_t)nx * ny * nz;
  double *b = (double *)malloc(sizeof(double) * N * 15);
  if (!b) return -1;
  const double *fs[3] = {f_n, f_n1, f_n2};
  double *rho[3], *ux[3], *uy[3], *uz[3];
  for (int m = 0; m < 3; ++m) {
    rho[m] = b + (4 * m) * N;
    ux[m] = b + (4 * m + 1) * N;
    uy[m] = b + (4 * m + 2) * N;
    uz[m] = b + (4 * m + 3) * N;
    orc3_moments(q, nx, ny, nz, kind, F0, kf, alpha, fs[m], rho[m], ux[m], uy[m], uz[m],
                 m == 0 ? b + 12 * N : NULL, m == 0 ? b + 13 * N : NULL,
                 m == 0 ? b + 14 * N : NULL);
  }
  int rc = orc3_terms(nx, ny, nz, tau, (const double *const *)rho, (const double *const *)ux,
                      (const double *const *)uy, (const double *const *)uz, b + 12 * N,
                      b + 13 * N, b + 14 * N, terms);
  free(b);
  return rc;
}

/* Mean of A over the L x L x L box with lower corner (x0, y0, z0), periodic. */
double orc3_box_mean(int nx, int ny, int nz, const double *A, int x0, int y0, int z0, int L) {
  double s = 0.0;
  for (int dz = 0; dz < L; ++dz)
    for (int dy = 0; dy < L; ++dy)
      for (int dx = 0; dx < L; ++dx)
        s += A[((size_t)wrap3(z0 + dz, nz) * ny + wrap3(y0 + dy, ny)) * nx + wrap3(x0 + dx, nx)];
  return s / ((double)L * L * L);
}

static double delta3(const double *b, int nrhs) {
  double lhs = b[0], sum = 0.0, mx = 0.0;
  for (int i = 1; i <= nrhs; ++i) {
    sum += b[i];
    if (fabs(b[i]) > mx) mx = fabs(b[i]);
  }
  double num = fabs(sum - lhs);
  if (mx == 0.0) return num == 0.0 ? 0.0 : INFINITY;
  return num / mx;
}

/* Statistics of the 15 box quantities [delta^E, delta^O, 13 terms] per size
 * (eqs. (12), (13); mean, population std), boxes at every periodic origin
 * (origins == NULL) or at the n_origins triples (x0, y0, z0); sizes that do
 * not fit give NaN.  per_box (nullable): [iL][box][15]. */
int orc3_balance_stats(int nx, int ny, int nz, const double *T, const int *Ls, int nL,
                       const int *origins, int n_origins, double *stats, double *per_box) {
  size_t N = (size_t)nx * ny * nz;
  int nb = origins ? n_origins : (int)N;
  double *vals = (double *)malloc(sizeof(double) * 15 * (size_t)nb);
  if (!vals) return -1;
  for (int iL = 0; iL < nL; ++iL) {
    int L = Ls[iL];
    double *st = stats + (size_t)iL * 30;
    if (L < 1 || L > nx || L > ny || L > nz) {
      for (int q = 0; q < 30; ++q) st[q] = NAN;
      continue;
    }
    for (int bx = 0; bx < nb; ++bx) {
      int x0, y0, z0;
      if (origins) {
        x0 = origins[3 * bx];
        y0 = origins[3 * bx + 1];
        z0 = origins[3 * bx + 2];
      } else {
        x0 = bx % nx;
        y0 = (bx / nx) % ny;
        z0 = bx / (nx * ny);
      }
      double v[13];
      for (int q = 0; q < 13; ++q) v[q] = orc3_box_mean(nx, ny, nz, T + (size_t)q * N, x0, y0, z0, L);
      double *o = vals + (size_t)bx * 15;
      o[0] = delta3(v, 5);
      o[1] = delta3(v + 6, 6);
      for (int q = 0; q < 13; ++q) o[2 + q] = v[q];
    }
    for (int q = 0; q < 15; ++q) {
      double m = 0.0, var = 0.0;
      for (int bx = 0; bx < nb; ++bx) m += vals[(size_t)bx * 15 + q];
      m /= nb;
      for (int bx = 0; bx < nb; ++bx) {
        double d = vals[(size_t)bx * 15 + q] - m;
        var += d * d;
      }
      st[2 * q] = m;
      st[2 * q + 1] = sqrt(var / nb);
    }
    if (per_box) memcpy(per_box + (size_t)iL * nb * 15, vals, sizeof(double) * 15 * nb);
  }
  free(vals);
  return 0;
}
