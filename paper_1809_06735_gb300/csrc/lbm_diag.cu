// Sub-volume energy/enstrophy balance diagnostic of Tauzin et al. (2018):
// the local terms of eqs. (8)-(11) in 2D with the eq. (18) 8th-order
// centred differences and the eq. (17) BDF2 time derivative, their L x L box
// averages through summed-area tables (O(1) per box and size), the balancing
// errors of eqs. (12), (13) and their statistics per box size.
//
// Precision.  Inputs are moment snapshots (rho, j_x, j_y): FP64 [3][ny*nx],
// or for FP32 storage the compensated FP32 pairs (hi, lo) of rho - rho0,
// j_x, j_y, [3][2][ny*nx], whose sums are the FP64 moments.  The term
// fields are computed in T = double (FP64 handles, or on request) or
// T = float (FP32 handles): GB300 executes FP64 at a small
// fraction of its FP32 rate, and the FP32 variant keeps its accuracy by
// forming every cancelling quantity from FP64 differences first -- the time
// differences u^n - u^{n-1} (so E and Omega differences, hence the eq. (17)
// derivatives, carry relative FP32 error of the difference, not of E), and
// the pressure gradient from rho - rho_ref.  Both variants use the same
// formulas.
// The summed-area tables are exact 64-bit fixed point: each field is scaled
// by a power of two 2^e chosen from its largest magnitude so that any
// partial sum stays below 2^62, rounded to integers once, and summed in
// integer arithmetic; a box sum is then exact (the only error is the one
// rounding of each cell, 2^-e, at most 2^-36 of the field's largest value on
// a 8192^2 grid).  Box means, balancing errors and statistics are formed in
// MT = double or float, again by handle precision; every block partial and
// final statistic is FP64 and block-deterministic.
//
// Batching.  The balance diagnostic of a group of members runs as ten
// launches in all (four term passes, scale exponents, the strip sums and
// the table builder, query constants, box query, statistics), blockIdx.z
// (or the CTA index of the
// per-job kernels) selecting the member; each member has its own field slot
// and partials slot.
//
// Field slot (doubles of N = nx*ny cells): slots 0..2 a temporary snapshot,
// slots 3.. the term-stage fields (each slot holds N values of T), then the
// int64 tables of (nx+1)(ny+1) records of 12 (13) interleaved fields.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

enum Field {
  U0X = 0, U0Y, DU01X, DU01Y, DU12X, DU12Y, DRHO, R0, FXR, FYR, A1, A2, WW, B1, B2, C1, C2,
  G1, G2, G3, K1, K2,
  T0,  // T0..T11: term fields 0..11 (term 12, vortex stretching, is 0 in 2D);
       // T0 + 12: |u|^2 (the sub-volume Mach number of eq. (20))
  NF = T0 + 13
};
constexpr int kSnapSlots = 3;
constexpr int kNT = 13;  // fields with a summed-area table: 12 terms, |u|^2
static_assert(kSnapSlots + NF + kNT <= kDiagFields, "scratch too small");

struct Grid {
  int nx, ny;
  double nu, alpha, rho_ref;
  const double *fxt, *fyt;  // F_ext,x(y), F_ext,y(x)
  // force kind 2: shell force [2][N], trig tables, damping coefficients
  const double *ft64, *trig64, *damp;
  const double *nu_field;  // local viscosity per cell (variable viscosity), else NULL
};

// External force (drag excluded) at cell (x, y): the separable tables, or
// for force kind 2 the shell force plus the damping of eq. (16).
__device__ __forceinline__ void ext_force(const Grid &g, int x, int y, double &fx, double &fy) {
  if (g.ft64) {
    double rx, ry;
    damping_at<double, double>(g.damp, g.trig64, g.nx, g.ny, x, y, rx, ry);
    const size_t c = (size_t)y * g.nx + x, N = (size_t)g.nx * g.ny;
    fx = g.ft64[c] + rx;
    fy = g.ft64[N + c] + ry;
  } else {
    fx = g.fxt[y];
    fy = g.fyt[x];
  }
}

template <typename T>
__host__ __device__ inline T *fld(double *base, int k, size_t N) {
  return reinterpret_cast<T *>(base + (size_t)(kSnapSlots + k) * N);
}
__host__ __device__ inline long long *sat_base(double *base, size_t N) {
  return reinterpret_cast<long long *>(base + (size_t)(kSnapSlots + NF) * N);
}
// The tables are the exclusive prefixes P_f(x, y) = sum over x' < x, y' < y
// of field f for 0 <= x <= nx, 0 <= y <= ny (row 0 and column 0 are zero),
// interleaved by field: record (x, y) holds the nF fields' values at
// ((y (nx + 1) + x) nF + f), so the corner of a box is one or two sectors
// for a whole balance instead of one sector per field.
__host__ __device__ inline size_t sat_stride(int nx, int ny) {
  return (size_t)(nx + 1) * (size_t)(ny + 1);
}

__device__ __forceinline__ int wr(int i, int n) {
  if (n >= 4) return i < 0 ? i + n : (i >= n ? i - n : i);
  return wrapi(i, n);
}

// Wrapped neighbour offsets of one cell, computed once and shared by every
// stencil of the cell: xo[d+4] = (x + d) mod nx, yo[d+4] = ((y + d) mod ny) nx.
struct Nb {
  int xo[9], yo[9];
};
__device__ __forceinline__ Nb make_nb(const Grid &g, int x, int y) {
  Nb nb;
#pragma unroll
  for (int d = -4; d <= 4; ++d) {
    nb.xo[d + 4] = wr(x + d, g.nx);
    nb.yo[d + 4] = wr(y + d, g.ny) * g.nx;
  }
  return nb;
}

// Eq. (18) in x and y (dx = 1), periodic, in the paired form
// 4/5 (A+1 - A-1) - 1/5 (A+2 - A-2) + 4/105 (A+3 - A-3) - 1/280 (A+4 - A-4).
template <typename T>
__device__ __forceinline__ T Dx(const T *A, const Nb &nb) {
  const T *r = A + nb.yo[4];
  return T(0.8) * (r[nb.xo[5]] - r[nb.xo[3]]) - T(0.2) * (r[nb.xo[6]] - r[nb.xo[2]]) +
         T(4.0 / 105.0) * (r[nb.xo[7]] - r[nb.xo[1]]) -
         T(1.0 / 280.0) * (r[nb.xo[8]] - r[nb.xo[0]]);
}
template <typename T>
__device__ __forceinline__ T Dy(const T *A, const Nb &nb) {
  const T *c = A + nb.xo[4];
  return T(0.8) * (c[nb.yo[5]] - c[nb.yo[3]]) - T(0.2) * (c[nb.yo[6]] - c[nb.yo[2]]) +
         T(4.0 / 105.0) * (c[nb.yo[7]] - c[nb.yo[1]]) -
         T(1.0 / 280.0) * (c[nb.yo[8]] - c[nb.yo[0]]);
}

constexpr int kQStats = 14;  // per balance: [delta, delta^2, (d_k, d_k^2) for its 6 fields]

// Per (size, field) constants of the query, computed once: the field mean,
// the factor from a quantized sum to a box mean, and the quantized sum a box
// of the mean value would have (so box deviations are exact integers).
struct QConst {
  double mean_d, coef_d;
  float mean_f, coef_f;
  long long mq;
  template <typename MT>
  __device__ MT mean() const;
  template <typename MT>
  __device__ MT coef() const;
};
template <> __device__ double QConst::mean<double>() const { return mean_d; }
template <> __device__ float QConst::mean<float>() const { return mean_f; }
template <> __device__ double QConst::coef<double>() const { return coef_d; }
template <> __device__ float QConst::coef<float>() const { return coef_f; }
constexpr int kQConstDoubles = kDiagMaxL * kNT * (int)(sizeof(QConst) / sizeof(double));
constexpr int kMaxQueryBlocks = 256;  // CTAs per (job, size, balance)

// Per-job partials slot, in 8-byte words: [0, 40) scale factors 2^e,
// 2^-e and the exponents e of the kNT tables; the per-size query constants
// [size][kNT]; the query CTA partials [size][3 groups][CTA][kQStats]; then
// the CTA maxima of the kNT fields, [kNT][CTAs of the cell grid].
constexpr size_t kPartScales = 0;
constexpr size_t kPartConsts = 40;
constexpr size_t kPartQuery = kPartConsts + kQConstDoubles;
constexpr size_t kPartMax = kPartQuery + (size_t)kDiagMaxL * 3 * kMaxQueryBlocks * kQStats;
__host__ __device__ constexpr size_t inv_scale(int f) { return kPartScales + kNT + f; }
__host__ __device__ constexpr size_t exps_at() { return kPartScales + 2 * kNT; }

#define CELL_INDEX                                        \
  const int x = blockIdx.x * blockDim.x + threadIdx.x;    \
  const int y = blockIdx.y * blockDim.y + threadIdx.y;    \
  if (x >= g.nx || y >= g.ny) return;                     \
  const size_t c = (size_t)y * g.nx + x;

// Cell passes of the batched diagnostic: CTAs of 32 x 8 cells, blockIdx.z
// the job.  A CTA wholly outside its job's grid returns at once; threads
// past a ragged edge stay (valid = false) for the CTA-wide reductions.
#define JOB_CELLS                                                            \
  const DiagJob &J = jobs[blockIdx.z];                                       \
  if ((int)(blockIdx.x * 32) >= J.nx || (int)(blockIdx.y * 8) >= J.ny) return; \
  const Grid g = job_grid(J);                                                \
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y; \
  const bool valid = x < g.nx && y < g.ny;                                   \
  const size_t N = (size_t)g.nx * g.ny, c = (size_t)y * g.nx + x;            \
  double *base = J.base;                                                     \
  const int nbx = (g.nx + 31) / 32, nblk = nbx * ((g.ny + 7) / 8);           \
  const int blk = blockIdx.y * nbx + blockIdx.x;

__device__ __forceinline__ Grid job_grid(const DiagJob &J) {
  Grid g;
  g.nx = J.nx;
  g.ny = J.ny;
  g.nu = J.nu;
  g.alpha = J.alpha;
  g.rho_ref = J.rho_ref;
  g.fxt = J.fxt;
  g.fyt = J.fyt;
  g.ft64 = nullptr;  // kind 2 is handled per level in k_prep
  g.trig64 = nullptr;
  g.damp = nullptr;
  g.nu_field = nullptr;  // the job's own per-cell viscosity (k_grad)
  return g;
}

template <typename T>
struct AbsBits;  // |v| as an unsigned integer that orders like |v|
template <>
struct AbsBits<float> {
  using U = unsigned;
  __device__ static U of(float v) {
    const U b = __float_as_uint(v) & 0x7fffffffu;
    return b > 0x7f800000u ? 0u : b;  // NaN counts as 0, as fmax does
  }
  __device__ static U warp_max(U b) { return __reduce_max_sync(0xffffffffu, b); }
  __device__ static double value(U b) { return (double)__uint_as_float(b); }
};
template <>
struct AbsBits<double> {
  using U = unsigned long long;
  __device__ static U of(double v) {
    const U b = (U)__double_as_longlong(v) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0ull : b;
  }
  __device__ static U warp_max(U b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const U n = __shfl_xor_sync(0xffffffffu, b, o);
      b = n > b ? n : b;
    }
    return b;
  }
  __device__ static double value(U b) { return __longlong_as_double((long long)b); }
};

// Row f of the CTA maxima of term field f (bit patterns of |T_f|).
template <typename T>
__device__ __forceinline__ typename AbsBits<T>::U *max_part(const DiagJob &J) {
  return reinterpret_cast<typename AbsBits<T>::U *>(J.part + kPartMax);
}

// Largest |v| over the CTA of K term fields (fields f[k]), stored at the
// CTA's slot of each field's row of maxima.  Every thread of the CTA calls it.
template <typename T, int K>
__device__ __forceinline__ void block_absmax(const T (&v)[K], const int (&f)[K],
                                             const DiagJob &J, int blk, int nblk) {
  using AB = AbsBits<T>;
  __shared__ typename AB::U sh[K][8];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const typename AB::U b = AB::warp_max(AB::of(v[k]));
    if (threadIdx.x == 0) sh[k][threadIdx.y] = b;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (threadIdx.y == 0 && threadIdx.x == k) {
      typename AB::U m = sh[k][0];
      for (int i = 1; i < 8; ++i) m = sh[k][i] > m ? sh[k][i] : m;
      max_part<T>(J)[(size_t)f[k] * nblk + blk] = m;
    }
  }
}

// Pass 0 (pointwise).  u = (j + F/2)/rho with F = F_ext - alpha j, i.e.
// rho u = m = (1 - alpha/2) j + F_ext/2.  Differences between levels:
// m^0 - m^1 = (1 - alpha/2)(j^0 - j^1), and
// u^0 - u^1 = (dm - u^0 drho) / rho^1  (exact identity).
// E^0 - E^1 = [drho |u^0|^2 + rho^1 du . (2 u^0 - du)] / 2, and
// LHS^E = (3 (E^0 - E^1) - (E^1 - E^2)) / 2 = eq. (17).
// The three snapshot levels of one cell: their FP64 values where the
// snapshots are FP64, and level differences formed without cancellation.
template <typename T, bool PAIRS>
struct Levels {
  T dr01, dr12, djx01, djy01, djx12, djy12;  // level differences n-(n-1), (n-1)-(n-2)
  T r0, r1, r2, jx0, jy0, drho;              // drho = rho^n - rho_ref
};

// FP64 snapshots [3][N]: differences in FP64, rounded once to T.
template <typename T>
__device__ __forceinline__ Levels<T, false> levels(const DiagJob &J, size_t N, size_t c) {
  const double *s0 = J.s0, *s1 = J.s1, *s2 = J.s2;
  const double r0d = s0[c], r1d = s1[c], r2d = s2[c];
  const double jx0d = s0[N + c], jy0d = s0[2 * N + c];
  const double jx1d = s1[N + c], jy1d = s1[2 * N + c];
  Levels<T, false> v;
  v.dr01 = (T)(r0d - r1d);
  v.dr12 = (T)(r1d - r2d);
  v.djx01 = (T)(jx0d - jx1d);
  v.djy01 = (T)(jy0d - jy1d);
  v.djx12 = (T)(jx1d - s2[N + c]);
  v.djy12 = (T)(jy1d - s2[2 * N + c]);
  v.r0 = (T)r0d;
  v.r1 = (T)r1d;
  v.r2 = (T)r2d;
  v.jx0 = (T)jx0d;
  v.jy0 = (T)jy0d;
  v.drho = (T)(r0d - J.rho_ref);
  return v;
}

// Compensated FP32 pairs [3][2][N] of (rho - rho0, j_x, j_y), rho0 = rho_ref:
// T = float forms each difference as (hi - hi') + (lo - lo') (relative error
// of the difference a few FP32 ulps, no FP64 instruction); T = double
// evaluates hi + lo in FP64 first (the exact compensated sums) and proceeds
// as from FP64 snapshots.
template <typename T>
__device__ __forceinline__ Levels<T, true> levels_pairs(const DiagJob &J, size_t N, size_t c) {
  const float *p[3] = {reinterpret_cast<const float *>(J.s0),
                       reinterpret_cast<const float *>(J.s1),
                       reinterpret_cast<const float *>(J.s2)};
  float hi[3][3], lo[3][3];  // [level][moment]
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      hi[k][q] = p[k][(size_t)(2 * q) * N + c];
      lo[k][q] = p[k][(size_t)(2 * q + 1) * N + c];
    }
  Levels<T, true> v;
  if constexpr (sizeof(T) == 4) {
    auto dif = [&](int q, int a, int b) { return (hi[a][q] - hi[b][q]) + (lo[a][q] - lo[b][q]); };
    v.dr01 = dif(0, 0, 1);
    v.dr12 = dif(0, 1, 2);
    v.djx01 = dif(1, 0, 1);
    v.djy01 = dif(2, 0, 1);
    v.djx12 = dif(1, 1, 2);
    v.djy12 = dif(2, 1, 2);
    const float rho0 = J.rho_ref_f;
    v.drho = hi[0][0] + lo[0][0];
    v.r0 = rho0 + v.drho;
    v.r1 = rho0 + (hi[1][0] + lo[1][0]);
    v.r2 = rho0 + (hi[2][0] + lo[2][0]);
    v.jx0 = hi[0][1] + lo[0][1];
    v.jy0 = hi[0][2] + lo[0][2];
  } else {
    double d[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int q = 0; q < 3; ++q) d[k][q] = (double)hi[k][q] + (double)lo[k][q];
    const double r0d = J.rho_ref + d[0][0], r1d = J.rho_ref + d[1][0],
                 r2d = J.rho_ref + d[2][0];
    v.dr01 = r0d - r1d;
    v.dr12 = r1d - r2d;
    v.djx01 = d[0][1] - d[1][1];
    v.djy01 = d[0][2] - d[1][2];
    v.djx12 = d[1][1] - d[2][1];
    v.djy12 = d[1][2] - d[2][2];
    v.r0 = r0d;
    v.r1 = r1d;
    v.r2 = r2d;
    v.jx0 = d[0][1];
    v.jy0 = d[0][2];
    v.drho = r0d - J.rho_ref;
  }
  return v;
}

// The 15 pointwise fields of pass 0 of one cell, in the order of kPrepField.
template <typename T>
struct PrepOut {
  T v[15];
};
__device__ constexpr int kPrepField[15] = {U0X, U0Y, DU01X, DU01Y, DU12X, DU12Y, DRHO, R0, FXR,
                                           FYR, A1, A2, T0 + 0, T0 + 3, T0 + 12};

// Pass 0 arithmetic of one cell from its levels, alpha, the external force
// at level n and the force's changes between levels (see k_prep).
template <typename T, bool PAIRS>
__device__ __forceinline__ PrepOut<T> prep_point(const Levels<T, PAIRS> &L, T a, T fex, T fey,
                                                 T dfx01, T dfy01, T dfx12, T dfy12) {
  const T ca = T(1) - T(0.5) * a;
  const T Fx = fex - a * L.jx0, Fy = fey - a * L.jy0;
  const T u0 = (L.jx0 + T(0.5) * Fx) / L.r0, v0 = (L.jy0 + T(0.5) * Fy) / L.r0;
  // m^n - m^{n-1} = (1 - alpha/2)(j^n - j^{n-1}) + (F_ext^n - F_ext^{n-1})/2
  const T du01 = (ca * L.djx01 + T(0.5) * dfx01 - u0 * L.dr01) / L.r1;
  const T dv01 = (ca * L.djy01 + T(0.5) * dfy01 - v0 * L.dr01) / L.r1;
  const T u1 = u0 - du01, v1 = v0 - dv01;
  const T du12 = (ca * L.djx12 + T(0.5) * dfx12 - u1 * L.dr12) / L.r2;
  const T dv12 = (ca * L.djy12 + T(0.5) * dfy12 - v1 * L.dr12) / L.r2;
  const T q0 = u0 * u0 + v0 * v0, q1 = u1 * u1 + v1 * v1;
  const T dE01 = T(0.5) * (L.dr01 * q0 +
                           L.r1 * (du01 * (T(2) * u0 - du01) + dv01 * (T(2) * v0 - dv01)));
  const T dE12 = T(0.5) * (L.dr12 * q1 +
                           L.r2 * (du12 * (T(2) * u1 - du12) + dv12 * (T(2) * v1 - dv12)));
  const T E0 = T(0.5) * L.r0 * q0;
  PrepOut<T> o;
  o.v[0] = u0;
  o.v[1] = v0;
  o.v[2] = du01;
  o.v[3] = dv01;
  o.v[4] = du12;
  o.v[5] = dv12;
  o.v[6] = L.drho;
  o.v[7] = L.r0;
  o.v[8] = Fx / L.r0;
  o.v[9] = Fy / L.r0;
  o.v[10] = E0 * u0;
  o.v[11] = E0 * v0;
  o.v[12] = T(0.5) * (T(3) * dE01 - dE12);  // LHS^E
  o.v[13] = u0 * Fx + v0 * Fy;               // RHS^{E,3} = u . F
  o.v[14] = q0;                              // |u|^2
  return o;
}

// Pass 0 (pointwise).  u = (j + F/2)/rho with F = F_ext - alpha j, i.e.
// rho u = m = (1 - alpha/2) j + F_ext/2.  Differences between levels:
// m^0 - m^1 = (1 - alpha/2)(j^0 - j^1), and
// u^0 - u^1 = (dm - u^0 drho) / rho^1  (exact identity).
// E^0 - E^1 = [drho |u^0|^2 + rho^1 du . (2 u^0 - du)] / 2, and
// LHS^E = (3 (E^0 - E^1) - (E^1 - E^2)) / 2 = eq. (17).
template <typename T, bool PAIRS>
__global__ void __launch_bounds__(256) k_prep(const DiagJob *__restrict__ jobs) {
  JOB_CELLS;
  T lhs = 0, uf = 0, uu = 0;
  if (valid) {
    Levels<T, PAIRS> L;
    if constexpr (PAIRS)
      L = levels_pairs<T>(J, N, c);
    else
      L = levels<T>(J, N, c);
    // alpha, the external force at level n, and its changes between levels
    // (non-zero only for the time-dependent damping of force kind 2)
    T a, fex, fey, dfx01 = 0, dfy01 = 0, dfx12 = 0, dfy12 = 0;
    if (J.force_kind == 2) {
      a = (T)g.alpha;
      double r[3][2];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        damping_at<double, double>(J.dc[k], J.trig64, g.nx, g.ny, x, y, r[k][0], r[k][1]);
      fex = (T)(J.ft64[c] + r[0][0]);
      fey = (T)(J.ft64[N + c] + r[0][1]);
      dfx01 = (T)(r[0][0] - r[1][0]);
      dfy01 = (T)(r[0][1] - r[1][1]);
      dfx12 = (T)(r[1][0] - r[2][0]);
      dfy12 = (T)(r[1][1] - r[2][1]);
    } else if constexpr (PAIRS && sizeof(T) == 4) {
      a = J.alpha_f;
      fex = J.fxt_f[y];
      fey = J.fyt_f[x];
    } else {
      a = (T)g.alpha;
      fex = (T)g.fxt[y];
      fey = (T)g.fyt[x];
    }
    const PrepOut<T> o = prep_point<T, PAIRS>(L, a, fex, fey, dfx01, dfy01, dfx12, dfy12);
    lhs = o.v[12];
    uf = o.v[13];
    uu = o.v[14];
#pragma unroll
    for (int k = 0; k < 15; ++k) fld<T>(base, kPrepField[k], N)[c] = o.v[k];
  }
  const T mv[3] = {lhs, uf, uu};
  const int mf[3] = {0, 3, 12};
  block_absmax<T, 3>(mv, mf, J, blk, nblk);
}

// Pass 0 for FP32 pair snapshots and force kinds 0/1 with two consecutive
// cells per thread (nx % 4 == 0): 18 eight-byte loads of the level pairs and
// 15 eight-byte stores per thread, the same per-cell arithmetic as k_prep.
// CTA (32, 8) covers 64 x 8 cells, the cells of the one-cell CTAs 2 bx and
// 2 bx + 1: maxima in slot 2 bx, zero in 2 bx + 1.
__global__ void __launch_bounds__(256) k_prep2(const DiagJob *__restrict__ jobs) {
  const DiagJob &J = jobs[blockIdx.z];
  if ((int)(blockIdx.x * 64) >= J.nx || (int)(blockIdx.y * 8) >= J.ny) return;
  const int nx = J.nx, ny = J.ny;
  const int x = blockIdx.x * 64 + 2 * threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  const bool valid = x < nx && y < ny;
  const size_t N = (size_t)nx * ny, c = (size_t)y * nx + x;
  double *base = J.base;
  const int nbx = (nx + 31) / 32, nblk = nbx * ((ny + 7) / 8);
  const int blk = blockIdx.y * nbx + 2 * blockIdx.x;
  float m0 = 0.f, m3 = 0.f, m12 = 0.f;
  if (valid) {
    const float *p[3] = {reinterpret_cast<const float *>(J.s0),
                         reinterpret_cast<const float *>(J.s1),
                         reinterpret_cast<const float *>(J.s2)};
    float2 hi[3][3], lo[3][3];  // [level][moment], two cells
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        hi[k][q] = __ldg(reinterpret_cast<const float2 *>(p[k] + (size_t)(2 * q) * N + c));
        lo[k][q] = __ldg(reinterpret_cast<const float2 *>(p[k] + (size_t)(2 * q + 1) * N + c));
      }
    const float fex = J.fxt_f[y], fey2[2] = {J.fyt_f[x], J.fyt_f[x + 1]};
    const float rho0 = J.rho_ref_f, a = J.alpha_f;
    PrepOut<float> o[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      auto h = [&](int k, int q) { return i ? hi[k][q].y : hi[k][q].x; };
      auto l = [&](int k, int q) { return i ? lo[k][q].y : lo[k][q].x; };
      auto dif = [&](int q, int a1, int b1) { return (h(a1, q) - h(b1, q)) + (l(a1, q) - l(b1, q)); };
      Levels<float, true> L;  // as levels_pairs<float>
      L.dr01 = dif(0, 0, 1);
      L.dr12 = dif(0, 1, 2);
      L.djx01 = dif(1, 0, 1);
      L.djy01 = dif(2, 0, 1);
      L.djx12 = dif(1, 1, 2);
      L.djy12 = dif(2, 1, 2);
      L.drho = h(0, 0) + l(0, 0);
      L.r0 = rho0 + L.drho;
      L.r1 = rho0 + (h(1, 0) + l(1, 0));
      L.r2 = rho0 + (h(2, 0) + l(2, 0));
      L.jx0 = h(0, 1) + l(0, 1);
      L.jy0 = h(0, 2) + l(0, 2);
      o[i] = prep_point<float, true>(L, a, fex, fey2[i], 0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 15; ++k)
      *reinterpret_cast<float2 *>(fld<float>(base, kPrepField[k], N) + c) =
          make_float2(o[0].v[k], o[1].v[k]);
    m0 = fmaxf(fabsf(o[0].v[12]), fabsf(o[1].v[12]));
    m3 = fmaxf(fabsf(o[0].v[13]), fabsf(o[1].v[13]));
    m12 = fmaxf(fabsf(o[0].v[14]), fabsf(o[1].v[14]));
  }
  const float mv[3] = {m0, m3, m12};
  const int mf[3] = {0, 3, 12};
  block_absmax<float, 3>(mv, mf, J, blk, nblk);
  if (threadIdx.y == 0 && threadIdx.x < 3 && (blk % nbx) + 1 < nbx)
    max_part<float>(J)[(size_t)mf[threadIdx.x] * nblk + blk + 1] = 0u;
}

// Pass 1 (radius 4): vorticity w = D_x u_y - D_y u_x and its level
// differences, LHS^Omega = (3 (O^0 - O^1) - (O^1 - O^2))/2 with
// O^0 - O^1 = dw (2 w^0 - dw)/2; velocity gradients; RHS^{E,2}
// (grad p = grad(rho - rho_ref)/3), RHS^{E,4}, RHS^{O,2}, RHS^{O,3};
// fluxes for pass 2.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_grad(const DiagJob *__restrict__ jobs) {
  JOB_CELLS;
  T t2 = 0, t4 = 0, t6 = 0, t8 = 0, t9 = 0;
  if (valid) {
    const Nb nb = make_nb(g, x, y);
    const T *U = fld<T>(base, U0X, N), *V = fld<T>(base, U0Y, N);
    const T w0 = Dx(V, nb) - Dy(U, nb);
    const T dw01 = Dx(fld<T>(base, DU01Y, N), nb) - Dy(fld<T>(base, DU01X, N), nb);
    const T dw12 = Dx(fld<T>(base, DU12Y, N), nb) - Dy(fld<T>(base, DU12X, N), nb);
    const T w1 = w0 - dw01;
    const T dO01 = T(0.5) * dw01 * (T(2) * w0 - dw01);
    const T dO12 = T(0.5) * dw12 * (T(2) * w1 - dw12);
    t6 = T(0.5) * (T(3) * dO01 - dO12);  // LHS^Omega
    const T Om = T(0.5) * w0 * w0;
    const T dxu = Dx(U, nb), dyu = Dy(U, nb);
    const T dxv = Dx(V, nb), dyv = Dy(V, nb);
    const T u = U[c], v = V[c], r = fld<T>(base, R0, N)[c];
    const T sxx = T(2) * dxu, sxy = dyu + dxv, syy = T(2) * dyv;  // S_ij = d_j u_i + d_i u_j
    T nu;  // the local viscosity at time n (variable-viscosity collisions)
    if (J.nu_cell_d)
      nu = (T)J.nu_cell_d[c];
    else if (J.nu_cell_f)
      nu = (T)J.nu_cell_f[c];
    else if constexpr (sizeof(T) == 4)
      nu = J.nu_f;
    else
      nu = g.nu;
    const T nr = nu * r;
    const T *DR = fld<T>(base, DRHO, N);
    t2 = -(u * Dx(DR, nb) + v * Dy(DR, nb)) / T(3);
    t4 = -nr * (sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv);
    t8 = -Om * (dxu + dyv);
    t9 = w0 * (Dx(fld<T>(base, FYR, N), nb) - Dy(fld<T>(base, FXR, N), nb));
    fld<T>(base, T0 + 6, N)[c] = t6;
    fld<T>(base, T0 + 2, N)[c] = t2;
    fld<T>(base, T0 + 4, N)[c] = t4;
    fld<T>(base, T0 + 8, N)[c] = t8;
    fld<T>(base, T0 + 9, N)[c] = t9;
    fld<T>(base, WW, N)[c] = w0;
    fld<T>(base, B1, N)[c] = Om * u;
    fld<T>(base, B2, N)[c] = Om * v;
    fld<T>(base, C1, N)[c] = nr * (u * sxx + v * sxy);
    fld<T>(base, C2, N)[c] = nr * (u * sxy + v * syy);
    fld<T>(base, G1, N)[c] = nr * sxx;
    fld<T>(base, G2, N)[c] = nr * sxy;
    fld<T>(base, G3, N)[c] = nr * syy;
  }
  const T mv[5] = {t2, t4, t6, t8, t9};
  const int mf[5] = {2, 4, 6, 8, 9};
  block_absmax<T, 5>(mv, mf, J, blk, nblk);
}

// Pass 2 (radius 4): RHS^{E,1}, RHS^{E,5}, RHS^{O,1}; H_i = d_j(nu rho S_ij)/rho;
// RHS^{O,4} = H_x d_y w - H_y d_x w; products w H for pass 3.
template <typename T>
__global__ void __launch_bounds__(256) k_flux(const DiagJob *__restrict__ jobs) {
  JOB_CELLS;
  T t1 = 0, t5 = 0, t7 = 0, t10 = 0;
  if (valid) {
    const Nb nb = make_nb(g, x, y);
    const T r = fld<T>(base, R0, N)[c];
    t1 = -(Dx(fld<T>(base, A1, N), nb) + Dy(fld<T>(base, A2, N), nb));
    t5 = Dx(fld<T>(base, C1, N), nb) + Dy(fld<T>(base, C2, N), nb);
    t7 = -(Dx(fld<T>(base, B1, N), nb) + Dy(fld<T>(base, B2, N), nb));
    const T Hx = (Dx(fld<T>(base, G1, N), nb) + Dy(fld<T>(base, G2, N), nb)) / r;
    const T Hy = (Dx(fld<T>(base, G2, N), nb) + Dy(fld<T>(base, G3, N), nb)) / r;
    const T *W = fld<T>(base, WW, N);
    t10 = Hx * Dy(W, nb) - Hy * Dx(W, nb);
    const T w = W[c];
    fld<T>(base, T0 + 1, N)[c] = t1;
    fld<T>(base, T0 + 5, N)[c] = t5;
    fld<T>(base, T0 + 7, N)[c] = t7;
    fld<T>(base, T0 + 10, N)[c] = t10;
    fld<T>(base, K1, N)[c] = w * Hy;
    fld<T>(base, K2, N)[c] = w * Hx;
  }
  const T mv[4] = {t1, t5, t7, t10};
  const int mf[4] = {1, 5, 7, 10};
  block_absmax<T, 4>(mv, mf, J, blk, nblk);
}

// Pass 3 (radius 4): RHS^{O,5} = d_x (w H_y) - d_y (w H_x).
template <typename T>
__global__ void __launch_bounds__(256) k_curl(const DiagJob *__restrict__ jobs) {
  JOB_CELLS;
  T t11 = 0;
  if (valid) {
    const Nb nb = make_nb(g, x, y);
    t11 = Dx(fld<T>(base, K1, N), nb) - Dy(fld<T>(base, K2, N), nb);
    fld<T>(base, T0 + 11, N)[c] = t11;
  }
  const T mv[1] = {t11};
  const int mf[1] = {11};
  block_absmax<T, 1>(mv, mf, J, blk, nblk);
}

// ---------------------------------------------------------------------------
// FP32 term passes 1-3 with four consecutive cells per thread (nx % 4 == 0):
// the x-taps of a row come from three aligned float4 loads (x - 4, x, x + 4,
// wrapped; nx % 4 == 0 keeps the wrapped quadruples aligned) and the y-taps
// from one float4 per row, about a sixth of the load instructions of the
// one-cell kernels above.  Same formulas per cell.  CTA (bx, by) covers
// 128 x 8 cells, i.e. the cells of the one-cell CTAs 4 bx .. 4 bx + 3 in
// row by: it stores its maxima in slot 4 bx and zero in the other three.
// ---------------------------------------------------------------------------

#define JOB_CELLS4                                                           \
  const DiagJob &J = jobs[blockIdx.z];                                       \
  if ((int)(blockIdx.x * 128) >= J.nx || (int)(blockIdx.y * 8) >= J.ny) return; \
  const int nx = J.nx, ny = J.ny;                                            \
  const int x = blockIdx.x * 128 + 4 * threadIdx.x, y = blockIdx.y * 8 + threadIdx.y; \
  const bool valid = x < nx && y < ny;                                       \
  const size_t N = (size_t)nx * ny, c = (size_t)y * nx + x;                  \
  double *base = J.base;                                                     \
  const int nbx = (nx + 31) / 32, nblk = nbx * ((ny + 7) / 8);               \
  const int blk = blockIdx.y * nbx + 4 * blockIdx.x;

// Wrapped offsets of a thread's quadruple: the quadruples left and right of
// it, and the row offsets y + d for d = -4..4.
struct Nb4 {
  int xl, xr, yo[9];
};
__device__ __forceinline__ Nb4 make_nb4(int nx, int ny, int x, int y) {
  Nb4 nb;
  nb.xl = x >= 4 ? x - 4 : x - 4 + nx;
  nb.xr = x + 4 < nx ? x + 4 : x + 4 - nx;
#pragma unroll
  for (int d = -4; d <= 4; ++d) nb.yo[d + 4] = wr(y + d, ny) * nx;
  return nb;
}
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
  const float4 q = __ldg(reinterpret_cast<const float4 *>(p));  // read-only in the pass
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
// Eq. (18) along x for the four cells (paired form as Dx), and their values.
__device__ __forceinline__ void dx4(const float *A, const Nb4 &nb, int x, float (&d)[4],
                                    float (&ctr)[4]) {
  float a[12];
  const float *r = A + nb.yo[4];
  float t[4];
  ld4(r + nb.xl, t);
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = t[i];
  ld4(r + x, t);
#pragma unroll
  for (int i = 0; i < 4; ++i) a[4 + i] = ctr[i] = t[i];
  ld4(r + nb.xr, t);
#pragma unroll
  for (int i = 0; i < 4; ++i) a[8 + i] = t[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = 4 + i;
    d[i] = 0.8f * (a[k + 1] - a[k - 1]) - 0.2f * (a[k + 2] - a[k - 2]) +
           float(4.0 / 105.0) * (a[k + 3] - a[k - 3]) -
           float(1.0 / 280.0) * (a[k + 4] - a[k - 4]);
  }
}
// Eq. (18) along y for the four cells.
__device__ __forceinline__ void dy4(const float *A, const Nb4 &nb, int x, float (&d)[4]) {
  float m[9][4];
#pragma unroll
  for (int k = 0; k < 9; ++k)
    if (k != 4) ld4(A + nb.yo[k] + x, m[k]);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    d[i] = 0.8f * (m[5][i] - m[3][i]) - 0.2f * (m[6][i] - m[2][i]) +
           float(4.0 / 105.0) * (m[7][i] - m[1][i]) - float(1.0 / 280.0) * (m[8][i] - m[0][i]);
}

// The CTA maxima of K fields from per-thread maxima (NaN-ignoring, as the
// one-cell kernels), stored in slot blk and zero in slots blk + 1..3.
template <int K>
__device__ __forceinline__ void block_absmax4(const float (&v)[K], const int (&f)[K],
                                              const DiagJob &J, int blk, int nblk, int nbx) {
  block_absmax<float, K>(v, f, J, blk, nblk);
  if (threadIdx.y == 0 && threadIdx.x < 3 * K) {
    const int k = threadIdx.x / 3, o = 1 + threadIdx.x % 3;
    if ((blk % nbx) + o < nbx) max_part<float>(J)[(size_t)f[k] * nblk + blk + o] = 0u;
  }
}
__device__ __forceinline__ float absmax4(const float (&t)[4]) {
  return fmaxf(fmaxf(fabsf(t[0]), fabsf(t[1])), fmaxf(fabsf(t[2]), fabsf(t[3])));
}

__global__ void __launch_bounds__(256, 2) k_grad4(const DiagJob *__restrict__ jobs) {
  JOB_CELLS4;
  float m2 = 0, m4 = 0, m6 = 0, m8 = 0, m9 = 0;
  if (valid) {
    const Nb4 nb = make_nb4(nx, ny, x, y);
    const float *U = fld<float>(base, U0X, N), *V = fld<float>(base, U0Y, N);
    float dxu[4], dyu[4], dxv[4], dyv[4], u[4], v[4], w0[4], a[4], b[4], t[4];
    dx4(U, nb, x, dxu, u);
    dy4(U, nb, x, dyu);
    dx4(V, nb, x, dxv, v);
    dy4(V, nb, x, dyv);
#pragma unroll
    for (int i = 0; i < 4; ++i) w0[i] = dxv[i] - dyu[i];
    st4(fld<float>(base, WW, N) + c, w0);
    // LHS^Omega from the vorticity differences between levels
    dx4(fld<float>(base, DU01Y, N), nb, x, a, t);
    dy4(fld<float>(base, DU01X, N), nb, x, b);
    float dw01[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) dw01[i] = a[i] - b[i];
    dx4(fld<float>(base, DU12Y, N), nb, x, a, t);
    dy4(fld<float>(base, DU12X, N), nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float dw12 = a[i] - b[i], w1 = w0[i] - dw01[i];
      const float dO01 = 0.5f * dw01[i] * (2.f * w0[i] - dw01[i]);
      const float dO12 = 0.5f * dw12 * (2.f * w1 - dw12);
      t[i] = 0.5f * (3.f * dO01 - dO12);
    }
    st4(fld<float>(base, T0 + 6, N) + c, t);
    m6 = absmax4(t);
    // RHS^{E,2} = -u . grad p
    const float *DR = fld<float>(base, DRHO, N);
    dx4(DR, nb, x, a, t);
    dy4(DR, nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = -(u[i] * a[i] + v[i] * b[i]) / 3.f;
    st4(fld<float>(base, T0 + 2, N) + c, t);
    m2 = absmax4(t);
    // RHS^{O,3} = w curl(F/rho)
    dx4(fld<float>(base, FYR, N), nb, x, a, t);
    dy4(fld<float>(base, FXR, N), nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = w0[i] * (a[i] - b[i]);
    st4(fld<float>(base, T0 + 9, N) + c, t);
    m9 = absmax4(t);
    float r[4], nr[4];
    ld4(fld<float>(base, R0, N) + c, r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float nu = J.nu_cell_d ? (float)J.nu_cell_d[c + i]
                                   : (J.nu_cell_f ? J.nu_cell_f[c + i] : J.nu_f);
      nr[i] = nu * r[i];
    }
    float sxx[4], sxy[4], syy[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      sxx[i] = 2.f * dxu[i];
      sxy[i] = dyu[i] + dxv[i];
      syy[i] = 2.f * dyv[i];
      t[i] = -nr[i] * (sxx[i] * dxu[i] + sxy[i] * dyu[i] + sxy[i] * dxv[i] + syy[i] * dyv[i]);
    }
    st4(fld<float>(base, T0 + 4, N) + c, t);
    m4 = absmax4(t);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float Om = 0.5f * w0[i] * w0[i];
      t[i] = -Om * (dxu[i] + dyv[i]);
      a[i] = Om * u[i];
      b[i] = Om * v[i];
    }
    st4(fld<float>(base, T0 + 8, N) + c, t);
    m8 = absmax4(t);
    st4(fld<float>(base, B1, N) + c, a);
    st4(fld<float>(base, B2, N) + c, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = nr[i] * (u[i] * sxx[i] + v[i] * sxy[i]);
      b[i] = nr[i] * (u[i] * sxy[i] + v[i] * syy[i]);
    }
    st4(fld<float>(base, C1, N) + c, a);
    st4(fld<float>(base, C2, N) + c, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = nr[i] * sxx[i];
      b[i] = nr[i] * sxy[i];
      t[i] = nr[i] * syy[i];
    }
    st4(fld<float>(base, G1, N) + c, a);
    st4(fld<float>(base, G2, N) + c, b);
    st4(fld<float>(base, G3, N) + c, t);
  }
  const float mv[5] = {m2, m4, m6, m8, m9};
  const int mf[5] = {2, 4, 6, 8, 9};
  block_absmax4<5>(mv, mf, J, blk, nblk, nbx);
}

__global__ void __launch_bounds__(256, 3) k_flux4(const DiagJob *__restrict__ jobs) {
  JOB_CELLS4;
  float m1 = 0, m5 = 0, m7 = 0, m10 = 0;
  if (valid) {
    const Nb4 nb = make_nb4(nx, ny, x, y);
    float a[4], b[4], ctr[4], t[4];
    float r[4];
    ld4(fld<float>(base, R0, N) + c, r);
    dx4(fld<float>(base, A1, N), nb, x, a, ctr);
    dy4(fld<float>(base, A2, N), nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = -(a[i] + b[i]);
    st4(fld<float>(base, T0 + 1, N) + c, t);
    m1 = absmax4(t);
    dx4(fld<float>(base, C1, N), nb, x, a, ctr);
    dy4(fld<float>(base, C2, N), nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = a[i] + b[i];
    st4(fld<float>(base, T0 + 5, N) + c, t);
    m5 = absmax4(t);
    dx4(fld<float>(base, B1, N), nb, x, a, ctr);
    dy4(fld<float>(base, B2, N), nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = -(a[i] + b[i]);
    st4(fld<float>(base, T0 + 7, N) + c, t);
    m7 = absmax4(t);
    float Hx[4], Hy[4];
    const float *G2p = fld<float>(base, G2, N);
    dx4(fld<float>(base, G1, N), nb, x, a, ctr);
    dy4(G2p, nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) Hx[i] = (a[i] + b[i]) / r[i];
    dx4(G2p, nb, x, a, ctr);
    dy4(fld<float>(base, G3, N), nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) Hy[i] = (a[i] + b[i]) / r[i];
    const float *W = fld<float>(base, WW, N);
    float w[4];
    dx4(W, nb, x, a, w);
    dy4(W, nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = Hx[i] * b[i] - Hy[i] * a[i];
    st4(fld<float>(base, T0 + 10, N) + c, t);
    m10 = absmax4(t);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = w[i] * Hy[i];
    st4(fld<float>(base, K1, N) + c, t);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = w[i] * Hx[i];
    st4(fld<float>(base, K2, N) + c, t);
  }
  const float mv[4] = {m1, m5, m7, m10};
  const int mf[4] = {1, 5, 7, 10};
  block_absmax4<4>(mv, mf, J, blk, nblk, nbx);
}

__global__ void __launch_bounds__(256) k_curl4(const DiagJob *__restrict__ jobs) {
  JOB_CELLS4;
  float m11 = 0;
  if (valid) {
    const Nb4 nb = make_nb4(nx, ny, x, y);
    float a[4], b[4], ctr[4], t[4];
    dx4(fld<float>(base, K1, N), nb, x, a, ctr);
    dy4(fld<float>(base, K2, N), nb, x, b);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = a[i] - b[i];
    st4(fld<float>(base, T0 + 11, N) + c, t);
    m11 = absmax4(t);
  }
  const float mv[1] = {m11};
  const int mf[1] = {11};
  block_absmax4<1>(mv, mf, J, blk, nblk, nbx);
}

// ---------------------------------------------------------------------------
// Block-deterministic reductions
// ---------------------------------------------------------------------------

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

// The same block sum with the warp stage in the accumulation type MT: only
// one value per warp and quantity is widened to FP64 (GB300 runs FP64
// arithmetic and conversions at a small fraction of its FP32 rate).
template <int NQ, typename MT>
__device__ void block_sum_store_mt(MT (&v)[NQ], double *out /*[NQ]*/) {
  __shared__ double sh[NQ][32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    MT a = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = (double)a;
  }
  __syncthreads();
  if (tid < NQ) {
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a += sh[tid][k];
    out[tid] = a;
  }
}

// Sums nb partial rows of width nq (fixed order per thread: 8 threads per
// quantity take interleaved rows, then a fixed-order combination).
__global__ void k_sum_partials(const double *partials, int nb, int nq, double *out) {
  const int q = threadIdx.x >> 3, j = threadIdx.x & 7;
  __shared__ double sh[32][8];
  double a = 0.0;
  if (q < nq)
    for (int b = j; b < nb; b += 8) a += partials[(size_t)b * nq + q];
  if (q < 32) sh[q][j] = a;
  __syncthreads();
  if (j == 0 && q < nq) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += sh[q][k];
    out[q] = s;
  }
}

// ---------------------------------------------------------------------------
// Moments and whole-grid quantities (FP64)
// ---------------------------------------------------------------------------

__global__ void k_moments(Grid g, const double *snap, size_t N, double *rho, double *ux,
                          double *uy) {
  CELL_INDEX;
  const double r = snap[c], jx = snap[N + c], jy = snap[2 * N + c];
  double fex, fey;
  ext_force(g, x, y, fex, fey);
  const double Fx = fex - g.alpha * jx, Fy = fey - g.alpha * jy;
  if (rho) rho[c] = r;
  ux[c] = (jx + 0.5 * Fx) / r;
  uy[c] = (jy + 0.5 * Fy) / r;
}

__global__ void k_vorticity(Grid g, const double *ux, const double *uy, double *omega) {
  CELL_INDEX;
  const Nb nb = make_nb(g, x, y);
  omega[c] = Dx(uy, nb) - Dy(ux, nb);
}

__global__ void k_global(Grid g, const double *snap, const double *ux, const double *uy,
                         size_t N, double *partials) {
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  for (size_t c = (size_t)blockIdx.x * nthr + tid; c < N; c += (size_t)gridDim.x * nthr) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    const Nb nb = make_nb(g, x, y);
    const double r = snap[c], jx = snap[N + c], jy = snap[2 * N + c];
    double fex, fey;
    ext_force(g, x, y, fex, fey);
    const double Fx = fex - g.alpha * jx, Fy = fey - g.alpha * jy;
    const double u = ux[c], v = uy[c];
    const double dxu = Dx(ux, nb), dyu = Dy(ux, nb);
    const double dxv = Dx(uy, nb), dyv = Dy(uy, nb);
    const double w = dxv - dyu;
    const double sxx = 2 * dxu, sxy = dyu + dxv, syy = 2 * dyv;
    acc[0] += r;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += 0.5 * r * (u * u + v * v);
    acc[4] += 0.5 * w * w;
    acc[5] += u * Fx + v * Fy;
    const double nu = g.nu_field ? g.nu_field[c] : g.nu;
    acc[6] += nu * r * (sxx * dxu + sxy * dyu + sxy * dxv + syy * dyv);
  }
  block_sum_store<7>(acc, partials + (size_t)blockIdx.x * 7);
}

__global__ void k_global_scale(double *sums, size_t N) {
  const int q = threadIdx.x;
  if (q >= 3 && q < 7) sums[q] /= (double)N;
}

// ---------------------------------------------------------------------------
// Exact fixed-point summed-area tables
// ---------------------------------------------------------------------------

// Scale exponents, one CTA of 256 threads per (field, job): e_f with
// N * max|T_f| * 2^e_f < 2^62 (so every partial sum of the table fits in
// int64), capped so that 2^e_f is a finite float.  scales[f] = 2^e_f,
// scales[kNT + f] = 2^-e_f, and the exponent itself at exps_at() as int.
// nF: the number of fields with a table in this call (12, or 13 with |u|^2).
template <typename T>
__global__ void __launch_bounds__(256) k_scales(const DiagJob *__restrict__ jobs, int nF) {
  const DiagJob &J = jobs[blockIdx.y];
  const int f = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (f >= nF) return;
  const size_t N = (size_t)J.nx * J.ny;
  const int nblk = ((J.nx + 31) / 32) * ((J.ny + 7) / 8);
  const typename AbsBits<T>::U *mb = max_part<T>(J) + (size_t)f * nblk;
  typename AbsBits<T>::U b = 0;
  for (int i = threadIdx.x; i < nblk; i += 256) b = mb[i] > b ? mb[i] : b;
  b = AbsBits<T>::warp_max(b);
  __shared__ typename AbsBits<T>::U wmax[8];
  if (lane == 0) wmax[wid] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) b = wmax[w] > b ? wmax[w] : b;
    const double m = AbsBits<T>::value(b);
    int e = 0;
    if (m > 0.0 && m <= 1.7e308) {
      int ex, nbits = 0;
      frexp(m, &ex);  // m < 2^ex
      while (((size_t)1 << nbits) < N) ++nbits;
      e = 62 - nbits - ex;
      if (e > 120) e = 120;
    }
    J.part[kPartScales + f] = ldexp(1.0, e);
    J.part[inv_scale(f)] = ldexp(1.0, -e);
    reinterpret_cast<int *>(J.part + exps_at())[f] = e;
  }
}

// round(v * 2^e) for a float v with |v| 2^e < 2^62 (ties to even), without
// float-to-integer conversions (GB300 runs them at a fraction of the ALU
// rate): w = v 2^e is exact in FP32; below 2^23 adding 2^23 rounds w to an
// integer that the sum's significand bits hold; from 2^23 on w already is an
// integer, its significand shifted by the exponent.  NaN or Inf gives 0.
__device__ __forceinline__ long long quantize(float v, int e) {
  const float w = v * __int_as_float((e + 127) << 23);  // 2^e, -126 <= e <= 120
  const float aw = fabsf(w);
  long long q;
  if (aw < 8388608.0f) {
    q = __float_as_int(aw + 8388608.0f) - 0x4B000000;
  } else {
    const unsigned bits = __float_as_uint(aw);
    const int sh = (int)(bits >> 23) - 150;  // 0 .. 38 for |w| < 2^62
    q = sh < 40 ? (long long)((bits & 0x7fffffu) | 0x800000u) << sh : 0ll;
  }
  return w < 0.0f ? -q : q;
}
__device__ __forceinline__ long long quantize(double v, int e) {
  // v 2^e (a product by a power of two: exact, as ldexp), 2^e from its bits
  return __double2ll_rn(v * __longlong_as_double((long long)(e + 1023) << 52));
}
// FP64 terms are quantised once, by k_strip_sums, which stores each value's
// integer over the value itself (the same width); the later passes of the
// table read the integers (no FP64 work there: with one strip a small grid
// has few CTAs, and the FP64 pipe of an SM is narrow).  FP32 terms are
// quantised on the fly (integer arithmetic only).
template <typename T> struct QTerm { using type = T; };
template <> struct QTerm<double> { using type = long long; };
__device__ __forceinline__ long long q_term(float v, int e) { return quantize(v, e); }
__device__ __forceinline__ long long q_term(long long v, int) { return v; }

// Summed-area tables by strips of kStrip = 128 columns, 4 consecutive cells
// per lane (each term field read twice, each table record written once):
//   k_strip_sums  per (field, row), the quantised sums of the row's strips
//                 and their exclusive prefix: the part of the row left of
//                 each strip;
//   k_sat_tile    a CTA per strip with one warp per field walks down the
//                 rows: left part + warp scan of the strip's 128 cells +
//                 running column sum (registers) is the table row, staged in
//                 shared memory and written as whole interleaved records.
// The left parts, int64 [field][strip][row], live in the term stage's
// intermediate fields (U0X on), dead by then: nF * ny * ceil(nx/128) <= 13 N.
constexpr int kStrip = 128;

__device__ __forceinline__ long long *strip_base(double *base, size_t N) {
  return reinterpret_cast<long long *>(fld<double>(base, U0X, N));
}

// Cells x..x+3 of a term row (zero past nx): one 16-byte load per float
// quadruple (two per double) where the row allows.
__device__ __forceinline__ void load4(const float *r, int x, int nx, bool vec, float (&v)[4]) {
  if (vec && x + 3 < nx) {
    const float4 q = *reinterpret_cast<const float4 *>(r + x);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = x + k < nx ? r[x + k] : 0.f;
  }
}
__device__ __forceinline__ void load4(const double *r, int x, int nx, bool vec, double (&v)[4]) {
  if (vec && x + 3 < nx) {
    const double2 a = *reinterpret_cast<const double2 *>(r + x);
    const double2 b = *reinterpret_cast<const double2 *>(r + x + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = x + k < nx ? r[x + k] : 0.0;
  }
}

__device__ __forceinline__ void load4(const long long *r, int x, int nx, bool vec,
                                      long long (&v)[4]) {
  if (vec && x + 3 < nx) {
    const longlong2 a = *reinterpret_cast<const longlong2 *>(r + x);
    const longlong2 b = *reinterpret_cast<const longlong2 *>(r + x + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = x + k < nx ? r[x + k] : 0ll;
  }
}

template <typename T>
__device__ __forceinline__ bool vec_rows(const T *A, int nx) {
  return nx % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
}

// One warp per (row, field), 4 strips in flight; grid (ceil(ny/8), nF, G).
template <typename T>
__global__ void __launch_bounds__(256) k_strip_sums(const DiagJob *__restrict__ jobs) {
  constexpr int U = 4;
  const DiagJob &J = jobs[blockIdx.z];
  const int nx = J.nx, ny = J.ny, f = blockIdx.y, ns = (nx + kStrip - 1) / kStrip;
  const int lane = threadIdx.x & 31, y = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (y >= ny) return;  // whole warps
  const size_t N = (size_t)nx * ny;
  T *A = fld<T>(J.base, T0 + f, N);
  const bool vec = vec_rows(A, nx);
  A += (size_t)y * nx;
  const int e = reinterpret_cast<const int *>(J.part + exps_at())[f];
  long long *out = strip_base(J.base, N) + (size_t)f * ns * ny + y;
  long long acc = 0;  // lane 0: the row's sum left of the current strip
  for (int s0 = 0; s0 < ns; s0 += U) {
    T a[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (s0 + u < ns) load4(A, (s0 + u) * kStrip + 4 * lane, nx, vec, a[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (s0 + u >= ns) break;
      long long v = 0, q[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        q[k] = quantize(a[u][k], e);
        v += q[k];
      }
      if constexpr (sizeof(T) == 8) {  // the integers over the values
        long long *r = reinterpret_cast<long long *>(A);
        const int x = (s0 + u) * kStrip + 4 * lane;
        if (vec && x + 3 < nx) {
          *reinterpret_cast<longlong2 *>(r + x) = make_longlong2(q[0], q[1]);
          *reinterpret_cast<longlong2 *>(r + x + 2) = make_longlong2(q[2], q[3]);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (x + k < nx) r[x + k] = q[k];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) {
        out[(size_t)(s0 + u) * ny] = acc;
        acc += v;
      }
    }
  }
}

__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Row blocks: with few strips (a large single member), the rows of a strip
// are split into nrb blocks of rb_rows rows (a multiple of 32) walked by
// separate CTAs.  k_col_sums gives each (field, strip, block) the quantised
// column sums of its rows and the sum of its rows' left parts, after the
// left parts [field][strip][row] at colsum_base; a block's CTA starts its
// running column sums at what the blocks above it sum to, exactly (integer
// arithmetic), so the table is the same whatever the split.
__device__ __forceinline__ long long *colsum_base(double *base, size_t N, int nF, int ns, int ny) {
  return strip_base(base, N) + (size_t)nF * ns * ny;
}

// A CTA of NF warps (warp f = field f) per (strip, row block, job).
template <typename T, int NF>
__global__ void __launch_bounds__(NF * 32) k_col_sums(const DiagJob *__restrict__ jobs,
                                                      int rb_rows) {
  constexpr int R = sizeof(T) == 4 ? 8 : 4;
  const int f = threadIdx.x >> 5, lane = threadIdx.x & 31, s = blockIdx.x, rb = blockIdx.y;
  const int nrb = gridDim.y;
  const DiagJob &J = jobs[blockIdx.z];
  const int nx = J.nx, ny = J.ny, ns = (nx + kStrip - 1) / kStrip;
  const int ya = rb * rb_rows, yb = ya + rb_rows < ny ? ya + rb_rows : ny;
  if (s >= ns || ya >= ny) return;  // whole CTA
  const size_t N = (size_t)nx * ny;
  using Q = typename QTerm<T>::type;
  const Q *A = reinterpret_cast<const Q *>(fld<T>(J.base, T0 + f, N));
  const bool vec = vec_rows(A, nx);
  const int x = s * kStrip + 4 * lane;
  const int e = reinterpret_cast<const int *>(J.part + exps_at())[f];
  const long long *left = strip_base(J.base, N) + ((size_t)f * ns + s) * ny;
  long long c[4] = {0, 0, 0, 0}, ls = 0;
  for (int y0 = ya; y0 < yb; y0 += R) {
    Q a[R][4];
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (y0 + k < yb) load4(A + (size_t)(y0 + k) * nx, x, nx, vec, a[k]);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (y0 + k >= yb) break;
#pragma unroll
      for (int j = 0; j < 4; ++j) c[j] += q_term(a[k][j], e);
    }
  }
  for (int y = ya + lane; y < yb; y += 32) ls += left[y];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ls += __shfl_down_sync(0xffffffffu, ls, o);
  long long *cs = colsum_base(J.base, N, NF, ns, ny) + (((size_t)f * ns + s) * nrb + rb) * kStrip;
#pragma unroll
  for (int j = 0; j < 4; ++j) cs[4 * lane + j] = c[j];
  long long *lsum = colsum_base(J.base, N, NF, ns, ny) + (size_t)NF * ns * nrb * kStrip;
  if (lane == 0) lsum[((size_t)f * ns + s) * nrb + rb] = ls;
}

// A CTA of NF warps (warp f = field f) per (strip, row block, job); grid
// (ns, nrb, G) (nrb = 1: the whole strip; rb_rows then >= ny).
// Lane l holds columns x0 + 4l .. x0 + 4l + 3.  Each row is staged in one of
// two shared tiles [field][129] (column c at (c % 4) 32 + c / 4: conflict-free
// writes) and copied out as the consecutive words of its records, so one
// barrier per row suffices.
template <typename T, int NF>
__global__ void __launch_bounds__(NF * 32) k_sat_tile(const DiagJob *__restrict__ jobs,
                                                      int rb_rows) {
  constexpr int R = sizeof(T) == 4 ? 8 : 4;  // rows of loads in flight per warp
  constexpr int NT = NF * 32, TS = kStrip + 1;
  __shared__ long long tile[2][NF][TS];
  const int f = threadIdx.x >> 5, lane = threadIdx.x & 31, s = blockIdx.x, rb = blockIdx.y;
  const int nrb = gridDim.y;
  const DiagJob &J = jobs[blockIdx.z];
  const int nx = J.nx, ny = J.ny, ns = (nx + kStrip - 1) / kStrip;
  const int ya = rb * rb_rows, yb = ya + rb_rows < ny ? ya + rb_rows : ny;
  if (s >= ns || ya >= ny) return;  // whole CTA
  const int x0 = s * kStrip, x = x0 + 4 * lane;
  const int nw = (nx - x0 < kStrip ? nx - x0 : kStrip) * NF;  // record words per row
  const size_t N = (size_t)nx * ny, rs = (size_t)nx + 1;
  using Q = typename QTerm<T>::type;
  const Q *A = reinterpret_cast<const Q *>(fld<T>(J.base, T0 + f, N));
  const bool vec = vec_rows(A, nx);
  const long long *left = strip_base(J.base, N) + ((size_t)f * ns + s) * ny;
  long long *tab = sat_base(J.base, N);
  const int e = reinterpret_cast<const int *>(J.part + exps_at())[f];
  long long col[4] = {0, 0, 0, 0}, lf = 0;
  if (rb == 0) {
    for (int w = threadIdx.x; w < nw; w += NT) tab[(size_t)(x0 + 1) * NF + w] = 0;  // row 0
    if (s == 0 && threadIdx.x < NF) tab[threadIdx.x] = 0;
  } else {  // the rows above this block: left parts plus the strip's column prefix
    const long long *cs = colsum_base(J.base, N, NF, ns, ny) + ((size_t)f * ns + s) * nrb * kStrip;
    const long long *lsum =
        colsum_base(J.base, N, NF, ns, ny) + (size_t)NF * ns * nrb * kStrip + ((size_t)f * ns + s) * nrb;
    long long c[4] = {0, 0, 0, 0}, ls = 0;
    for (int b = 0; b < rb; ++b) {
#pragma unroll
      for (int j = 0; j < 4; ++j) c[j] += cs[(size_t)b * kStrip + 4 * lane + j];
      ls += lsum[b];
    }
    c[1] += c[0];
    c[2] += c[1];
    c[3] += c[2];
    const long long off = ls + warp_incl_scan(c[3], lane) - c[3];
#pragma unroll
    for (int j = 0; j < 4; ++j) col[j] = off + c[j];
  }
  for (int y0 = ya; y0 < yb; y0 += R) {
    if ((y0 & 31) == 0) lf = y0 + lane < ny ? left[y0 + lane] : 0;  // 32 rows' left parts
    Q a[R][4];
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (y0 + k < yb) load4(A + (size_t)(y0 + k) * nx, x, nx, vec, a[k]);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int y = y0 + k;
      const long long l = __shfl_sync(0xffffffffu, lf, (y0 & 31) + k);
      if (y >= yb) break;  // the same for the whole CTA
      long long v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = q_term(a[k][j], e);
      v[1] += v[0];
      v[2] += v[1];
      v[3] += v[2];
      const long long off = l + warp_incl_scan(v[3], lane) - v[3];
      long long *t = tile[y & 1][f];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        col[j] += off + v[j];
        t[j * 32 + lane] = col[j];
      }
      __syncthreads();
      long long *out = tab + ((size_t)(y + 1) * rs + x0 + 1) * NF;
      for (int w = threadIdx.x; w < nw; w += NT) {
        const int c = w / NF, g = w - c * NF;
        out[w] = tile[y & 1][g][(c & 3) * 32 + (c >> 2)];
      }
      if (s == 0 && threadIdx.x < NF) tab[(size_t)(y + 1) * rs * NF + threadIdx.x] = 0;
    }
  }
}

// Exclusive prefix P(x, y) (0 <= x <= nx, 0 <= y <= ny) from a padded table;
// modular (unsigned) arithmetic: the periodic extension may exceed int64 in
// between, the box sum does not.
__device__ __forceinline__ unsigned long long Pex(const long long *S, int nx, int nF, int x,
                                                  int y) {
  return (unsigned long long)S[((size_t)y * (nx + 1) + x) * nF];
}
__device__ __forceinline__ unsigned long long Pext(const long long *S, int nx, int ny, int nF,
                                                   int x, int y) {
  const int qx = x >= nx, qy = y >= ny;
  const int xm = x - qx * nx, ym = y - qy * ny;
  unsigned long long v = Pex(S, nx, nF, xm, ym);
  if (qx) v += Pex(S, nx, nF, nx, ym);
  if (qy) v += Pex(S, nx, nF, xm, ny);
  if (qx && qy) v += Pex(S, nx, nF, nx, ny);
  return v;
}

template <typename MT>
__device__ __forceinline__ MT delta_of(MT lhs, MT sum, MT mx) {
  const MT num = fabs(sum - lhs);
  if (mx == MT(0)) return num == MT(0) ? MT(0) : MT(INFINITY);
  return num / mx;
}

// One CTA per job, one thread per (size, field); constants at [size][kNT].
__global__ void k_query_consts(const DiagJob *__restrict__ jobs, int nF) {
  const DiagJob &J = jobs[blockIdx.x];
  const int t = threadIdx.x;
  const int iL = t / kNT, k = t % kNT;
  if (iL >= J.nL || k >= nF) return;
  const int nx = J.nx, ny = J.ny;
  const size_t N = (size_t)nx * ny;
  const double area = (double)J.meta[8 * iL] * (double)J.meta[8 * iL];
  const long long total = sat_base(J.base, N)[(sat_stride(nx, ny) - 1) * nF + k];
  const double inv = J.part[inv_scale(k)];
  QConst q;
  q.mean_d = (double)total * inv / (double)N;
  q.coef_d = inv / area;
  q.mean_f = (float)q.mean_d;
  q.coef_f = (float)q.coef_d;
  q.mq = __double2ll_rn((double)total * area / (double)N);
  reinterpret_cast<QConst *>(J.part + kPartConsts)[t] = q;
}

// 64-bit integer to the query precision.  The float version assembles the
// IEEE bits with integer instructions (leading-zero count, shift, round half
// up): GB300 issues integer-to-float conversions on its slow FP64 pipe.
template <typename MT>
__device__ __forceinline__ MT to_mt(long long v);
template <>
__device__ __forceinline__ double to_mt<double>(long long v) {
  return (double)v;
}
template <>
__device__ __forceinline__ float to_mt<float>(long long v) {
  // |v| = h 2^42 + m 2^21 + l with l, m < 2^21 and h <= 2^22: each piece is
  // exact in FP32 once its bits are placed in the mantissa of 2^23 and that
  // constant is subtracted; two fused multiply-adds of non-negative terms
  // combine them (at most one unit in the last place from the correctly
  // rounded value, the same for every call), the sign is applied last.  No
  // integer-to-float instruction: GB300 issues those at a small fraction of
  // the FP32 rate.
  const bool neg = v < 0;
  const unsigned long long a = neg ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const unsigned l = (unsigned)a & 0x1FFFFFu;
  const unsigned m = (unsigned)(a >> 21) & 0x1FFFFFu;
  const unsigned h = (unsigned)(a >> 42);
  const float fl = __uint_as_float(0x4B000000u | l) - 8388608.0f;
  const float fm = __uint_as_float(0x4B000000u | m) - 8388608.0f;
  const float fh = __uint_as_float(0x4B000000u | h) - 8388608.0f;
  const float r = fmaf(fh, 4398046511104.0f, fmaf(fm, 2097152.0f, fl));
  return neg ? -r : r;
}

// Bin of v among ne ascending edges: the number of edges <= v.
template <typename MT>
__device__ __forceinline__ int bin_of(MT v, const MT *edges, int ne) {
  int lo = 0, hi = ne;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (edges[mid] <= v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Block sum of the two balances' accumulators of a CTA whose even threads
// hold energy (group 0) and odd threads enstrophy (group 1) values: warp
// stage in MT over lanes of one parity, then a fixed-order sum over warps.
template <int NQ, typename MT>
__device__ void block_sum_store_pairs(MT (&v)[NQ], double *out0, double *out1) {
  __shared__ double sh[2][NQ][32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    MT a = v[q];
#pragma unroll
    for (int o = 16; o > 1; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane < 2) sh[lane][q][wid] = (double)a;
  }
  __syncthreads();
  if (tid < 2 * NQ) {
    const int g = tid / NQ, q = tid % NQ;
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a += sh[g][q][k];
    (g ? out1 : out0)[q] = a;
  }
}

// Grid (query CTAs, sizes, NZ x jobs), NZ = 1, or 2 with the distributions
// (EXT), blockIdx.z = NZ * job + part.  Part 0: thread pairs per box, the
// even thread the energy balance (fields 0..5: LHS^E, RHS^{E,1..5}), the odd
// one the enstrophy balance (fields 6..11: LHS^O, RHS^{O,1..5}; RHS^{O,6}
// is identically 0 in 2D and adds nothing), so the two read the halves of
// the same interleaved corner records; part 1 (EXT): one thread per box for
// the sub-volume Mach number (field 12, |u|^2).  Each thread walks its boxes
// (CTA c takes passes c, c + qb, ...) with the next origin prefetched:
// exact integer box sums of the group's fields, their deviations d_k from
// the field means, the box means, the balancing error (or Ma_V), and sums of
// d_k, d_k^2 and of the error's (or Ma_V's) deviation and its square; with
// EXT also a CTA histogram in shared memory, added to the global one with
// integer atomics (order-free, so deterministic).
template <typename MT, bool PER_BOX, bool EXT>
__global__ void __launch_bounds__(256, 3) k_query(const DiagJob *__restrict__ jobs, int nF,
                                               const int *__restrict__ origins,
                                               double *per_box, DiagDist ext) {
  constexpr int NZ = EXT ? 2 : 1;
  const DiagJob &J = jobs[blockIdx.z / NZ];
  const bool mpart = EXT && blockIdx.z % NZ == 1;
  const int iL = blockIdx.y;
  if (iL >= J.nL || (int)blockIdx.x >= J.qblocks) return;
  const int grp = mpart ? 2 : (int)(threadIdx.x & 1), k0 = 6 * grp;
  const int slot = mpart ? (int)threadIdx.x : (int)(threadIdx.x >> 1);
  const int per_pass = mpart ? 256 : 128;
  const int qb = J.qblocks;
  const int nx = J.nx, ny = J.ny;
  const int *meta = J.meta;
  const int L = meta[8 * iL], nb = meta[8 * iL + 1], ooff = meta[8 * iL + 2];
  const size_t N = (size_t)nx * ny;
  const size_t rs = (size_t)nx + 1;
  const long long *S = sat_base(J.base, N) + k0;
  const QConst *qc =
      reinterpret_cast<const QConst *>(J.part + kPartConsts) + (size_t)iL * kNT + k0;
  const int nfield = grp == 2 ? 1 : 6;
  __shared__ MT sedge[EXT ? kDiagMaxEdges : 1];
  __shared__ unsigned shist[2][EXT ? kDiagMaxEdges + 1 : 1];
  int ne = 0;
  if constexpr (EXT) {
    ne = mpart ? ext.n_mach : ext.n_delta;
    const double *e = mpart ? ext.mach_edges : ext.delta_edges;
    for (int i = threadIdx.x; i <= ne; i += blockDim.x) {
      if (i < ne) sedge[i] = (MT)e[i];
      shist[0][i] = 0u;
      shist[1][i] = 0u;
    }
    __syncthreads();
  }
  // group 2: deviations of Ma_V from the whole-grid value
  const MT ma_ref = EXT ? sqrt(fmax(qc[0].mean<MT>(), MT(0))) * MT(1.7320508075688772) : MT(0);
  MT s1[6], s2[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    s1[j] = MT(0);
    s2[j] = MT(0);
  }
  MT d1 = 0, d2 = 0;
  const int stride = qb * per_pass;
  int b = blockIdx.x * per_pass + slot;
  auto origin = [&](int i, int &x, int &y) {
    if (ooff >= 0) {
      x = origins[2 * (ooff + i)];
      y = origins[2 * (ooff + i) + 1];
    } else {
      x = i % nx;
      y = i / nx;
    }
  };
  int x0 = 0, y0 = 0;
  if (b < nb) origin(b, x0, y0);
  // all periodic origins in row-major order: the next origin is this one
  // advanced by the stride (no division per box)
  const int sdx = ooff < 0 ? stride % nx : 0, sdy = ooff < 0 ? stride / nx : 0;
  for (; b < nb; b += stride) {
    int xn = 0, yn = 0;  // the next box's origin, loaded ahead
    if (ooff < 0) {
      xn = x0 + sdx;
      yn = y0 + sdy;
      if (xn >= nx) {
        xn -= nx;
        ++yn;
      }
    } else if (b + stride < nb) {
      origin(b + stride, xn, yn);
    }
    const bool inside = x0 + L <= nx && y0 + L <= ny;
    MT lhs = 0, sum = 0, mx = 0;
    double *o = PER_BOX ? per_box + ((size_t)meta[8 * iL + 3] + b) * 15 : nullptr;
    // a non-wrapping box of a 12-field table: the six values of a corner are
    // 48 bytes at a 16-byte boundary, three vector loads per corner
    unsigned long long vs[6];
    const bool vec = nF == 12 && nfield == 6;
    if (vec && !inside) {
      // a box across the periodic edge: the prefix sum extended periodically
      // is a signed sum of at most 3 x 3 table corners, columns
      // {x0 + L, x0} or {nx, x0, x0 + L - nx} (and rows likewise); each
      // corner's six values are three 16-byte loads
      const int wx = x0 + L > nx, wy = y0 + L > ny;
      const int X[3] = {wx ? nx : x0 + L, x0, x0 + L - nx};
      const int Y[3] = {wy ? ny : y0 + L, y0, y0 + L - ny};
#pragma unroll
      for (int j = 0; j < 6; ++j) vs[j] = 0ull;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (k == 2 && !wy) break;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (i == 2 && !wx) break;
          const bool neg = (i == 1) != (k == 1);  // the x0 column and the y0 row subtract
          const longlong2 *c =
              reinterpret_cast<const longlong2 *>(S + ((size_t)Y[k] * rs + X[i]) * 12);
#pragma unroll
          for (int h = 0; h < 3; ++h) {
            const longlong2 a = c[h];
            const unsigned long long ax = (unsigned long long)a.x, ay = (unsigned long long)a.y;
            vs[2 * h] = neg ? vs[2 * h] - ax : vs[2 * h] + ax;
            vs[2 * h + 1] = neg ? vs[2 * h + 1] - ay : vs[2 * h + 1] + ay;
          }
        }
      }
    } else if (vec) {
      const long long *lo = S + ((size_t)y0 * rs + x0) * 12, *hi = lo + (size_t)L * rs * 12;
      const size_t dx = (size_t)L * 12;
      const longlong2 *c00 = reinterpret_cast<const longlong2 *>(lo);
      const longlong2 *c10 = reinterpret_cast<const longlong2 *>(lo + dx);
      const longlong2 *c01 = reinterpret_cast<const longlong2 *>(hi);
      const longlong2 *c11 = reinterpret_cast<const longlong2 *>(hi + dx);
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        const longlong2 a00 = c00[h], a10 = c10[h], a01 = c01[h], a11 = c11[h];
        vs[2 * h] = (unsigned long long)a11.x - (unsigned long long)a01.x -
                    (unsigned long long)a10.x + (unsigned long long)a00.x;
        vs[2 * h + 1] = (unsigned long long)a11.y - (unsigned long long)a01.y -
                        (unsigned long long)a10.y + (unsigned long long)a00.y;
      }
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (j >= nfield) break;
      const long long *Sk = S + j;
      unsigned long long bs;
      if (vec) {
        bs = vs[j];
      } else if (inside) {  // no periodic wrap: four direct corner loads
        const long long *lo = Sk + ((size_t)y0 * rs + x0) * nF, *hi = lo + (size_t)L * rs * nF;
        const size_t dx = (size_t)L * nF;
        bs = (unsigned long long)hi[dx] - (unsigned long long)hi[0] -
             (unsigned long long)lo[dx] + (unsigned long long)lo[0];
      } else {
        bs = Pext(Sk, nx, ny, nF, x0 + L, y0 + L) - Pext(Sk, nx, ny, nF, x0, y0 + L) -
             Pext(Sk, nx, ny, nF, x0 + L, y0) + Pext(Sk, nx, ny, nF, x0, y0);
      }
      const long long dq = (long long)(bs - (unsigned long long)qc[j].mq);
      const MT d = to_mt<MT>(dq) * qc[j].coef<MT>();
      const MT v = d + qc[j].mean<MT>();
      s1[j] += d;
      s2[j] += d * d;
      if (j == 0) {
        lhs = v;
      } else {
        sum += v;
        mx = fmax(mx, fabs(v));
      }
      if (PER_BOX) o[2 + k0 + j] = (double)v;
    }
    MT val;  // delta of the group's balance, or Ma_V
    if (EXT && grp == 2) {
      val = sqrt(fmax(lhs, MT(0))) * MT(1.7320508075688772);
      const MT dm = val - ma_ref;
      d1 += dm;
      d2 += dm * dm;
    } else {
      val = delta_of(lhs, sum, mx);
      d1 += val;
      d2 += val * val;
    }
    if constexpr (EXT) {
      if (val == val) atomicAdd(&shist[mpart ? 0 : grp][bin_of(val, sedge, ne)], 1u);
    }
    if (PER_BOX) {
      o[grp] = (double)val;
      if (grp == 1) o[14] = 0.0;
    }
    x0 = xn;
    y0 = yn;
  }
  MT acc[kQStats];
  acc[0] = d1;
  acc[1] = d2;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    acc[2 + 2 * j] = s1[j];
    acc[3 + 2 * j] = s2[j];
  }
  double *pq = J.part + kPartQuery;
  if (mpart)
    block_sum_store_mt<kQStats, MT>(acc, pq + (((size_t)iL * 3 + 2) * qb + blockIdx.x) * kQStats);
  else
    block_sum_store_pairs<kQStats, MT>(acc, pq + (((size_t)iL * 3 + 0) * qb + blockIdx.x) * kQStats,
                                       pq + (((size_t)iL * 3 + 1) * qb + blockIdx.x) * kQStats);
  if constexpr (EXT) {
    __syncthreads();
    const int ng = mpart ? 1 : 2;
    for (int g = 0; g < ng; ++g) {
      unsigned long long *h =
          ext.hist + ((size_t)meta[8 * iL + 4] * 3 + (mpart ? 2 : g)) * (kDiagMaxEdges + 1);
      for (int i = threadIdx.x; i <= ne; i += blockDim.x)
        if (shist[g][i]) atomicAdd(&h[i], (unsigned long long)shist[g][i]);
    }
  }
}

// Mean and population standard deviation of the 15 quantities per size,
// and with `mach` those of Ma_V.  Grid (sizes, jobs), 384 threads: 8 per
// (group, slot) sum interleaved block partials in a fixed order.
template <typename MT>
__global__ void k_stats_final(const DiagJob *__restrict__ jobs, double *stats, double *mach) {
  const DiagJob &J = jobs[blockIdx.y];
  const int iL = blockIdx.x;
  if (iL >= J.nL) return;
  const int nblocks = J.qblocks;
  const double *partials = J.part + kPartQuery;
  const QConst *consts = reinterpret_cast<const QConst *>(J.part + kPartConsts);
  const int q = threadIdx.x >> 3, j = threadIdx.x & 7;  // q = grp * 14 + slot
  const int ngrp = mach ? 3 : 2;
  __shared__ double sh[3 * kQStats][8];
  double a = 0.0;
  if (q < ngrp * kQStats) {
    const int grp = q / kQStats, slot = q % kQStats;
    for (int b = j; b < nblocks; b += 8)
      a += partials[(((size_t)iL * 3 + grp) * nblocks + b) * kQStats + slot];
    sh[q][j] = a;
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int nb = J.meta[8 * iL + 1];
  const size_t orow = (size_t)J.meta[8 * iL + 4];
  if (t < 15) {
    double mean = 0.0, sd = 0.0;
    if (t < 14) {
      int row;  // row of sh holding the (sum, sum of squares) pair
      double shift = 0.0;
      if (t < 2) {
        row = t * kQStats;
      } else {
        const int k = t - 2, grp = k / 6;
        row = grp * kQStats + 2 + 2 * (k % 6);
        shift = consts[(size_t)iL * kNT + k].mean_d;
      }
      double s1 = 0.0, s2 = 0.0;
      for (int m = 0; m < 8; ++m) {
        s1 += sh[row][m];
        s2 += sh[row + 1][m];
      }
      const double m1 = s1 / nb;
      mean = shift + m1;
      sd = sqrt(fmax(s2 / nb - m1 * m1, 0.0));
    }
    stats[(orow * 15 + t) * 2] = mean;
    stats[(orow * 15 + t) * 2 + 1] = sd;
  } else if (t == 32 && mach) {
    const int row = 2 * kQStats;
    double s1 = 0.0, s2 = 0.0;
    for (int m = 0; m < 8; ++m) {
      s1 += sh[row][m];
      s2 += sh[row + 1][m];
    }
    // the reference value the query subtracted, in the query precision
    const QConst &c = consts[(size_t)iL * kNT + 12];
    const double ref = (double)(sqrt(fmax(c.mean<MT>(), MT(0))) * MT(1.7320508075688772));
    const double m1 = s1 / nb;
    mach[orow * 2] = ref + m1;
    mach[orow * 2 + 1] = sqrt(fmax(s2 / nb - m1 * m1, 0.0));
  }
}

Grid grid_of(const Member &hm) {
  Grid g;
  g.nx = hm.nx;
  g.ny = hm.ny;
  g.nu = hm.nu;
  g.alpha = hm.alpha;
  g.rho_ref = hm.rho0;
  g.fxt = hm.fx_tab64;
  g.fyt = hm.fy_tab64;
  const bool k2 = hm.force_kind == 2;  // damping of the current state (Member::damp)
  g.ft64 = k2 ? hm.ft_tab64 : nullptr;
  g.trig64 = k2 ? hm.trig64 : nullptr;
  g.damp = k2 ? hm.damp : nullptr;
  g.nu_field = nullptr;
  return g;
}

dim3 cells_grid(const Grid &g, dim3 b) {
  return dim3((g.nx + b.x - 1) / b.x, (g.ny + b.y - 1) / b.y);
}

template <typename T, typename MT>
cudaError_t balance_launches(const DiagJob *jobs_host, const DiagJob *jobs, int G, bool pairs,
                             const int *origins, double *stats, double *per_box,
                             const DiagDist *dist, cudaStream_t s) {
  int nx = 1, ny = 1, nL = 1, qblocks = 1;
  for (int j = 0; j < G; ++j) {
    nx = std::max(nx, jobs_host[j].nx);
    ny = std::max(ny, jobs_host[j].ny);
    nL = std::max(nL, jobs_host[j].nL);
    qblocks = std::max(qblocks, jobs_host[j].qblocks);
  }
  const int nF = dist ? kNT : 12;  // |u|^2 gets a table only for Ma_V
  const dim3 cb(32, 8), cg((nx + 31) / 32, (ny + 7) / 8, G);
  bool quad = sizeof(T) == 4;  // four cells per thread where every job allows
  for (int j = 0; j < G && quad; ++j)
    quad = jobs_host[j].nx % 4 == 0 && (reinterpret_cast<uintptr_t>(jobs_host[j].base) & 15) == 0;
  bool pair2 = quad && pairs;  // two-cell pass 0: FP32 pairs, force kinds 0 and 1
  for (int j = 0; j < G && pair2; ++j) pair2 = jobs_host[j].force_kind != 2;
  if (pair2)
    k_prep2<<<dim3((nx + 63) / 64, (ny + 7) / 8, G), cb, 0, s>>>(jobs);
  else if (pairs)
    k_prep<T, true><<<cg, cb, 0, s>>>(jobs);
  else
    k_prep<T, false><<<cg, cb, 0, s>>>(jobs);
  if (quad) {
    const dim3 cg4((nx + 127) / 128, (ny + 7) / 8, G);
    k_grad4<<<cg4, cb, 0, s>>>(jobs);
    k_flux4<<<cg4, cb, 0, s>>>(jobs);
    k_curl4<<<cg4, cb, 0, s>>>(jobs);
  } else {
    k_grad<T><<<cg, cb, 0, s>>>(jobs);
    k_flux<T><<<cg, cb, 0, s>>>(jobs);
    k_curl<T><<<cg, cb, 0, s>>>(jobs);
  }
  k_scales<T><<<dim3(nF, G), 256, 0, s>>>(jobs, nF);
  const int ns = (nx + kStrip - 1) / kStrip;
  k_strip_sums<T><<<dim3((ny + 7) / 8, nF, G), 256, 0, s>>>(jobs);
  // row blocks when strips x jobs would leave SMs idle
  int rb_rows = ny, nrb = 1;
  {
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    }
    const long long ctas = (long long)ns * G;
    if (ctas < sms && ny >= 64) {
      long long want = (2LL * sms + ctas - 1) / ctas;
      if (want > ny / (ny >= 256 ? 64 : 32)) want = ny / (ny >= 256 ? 64 : 32);
      rb_rows = (int)(((ny + want - 1) / want + 31) / 32 * 32);
      nrb = (ny + rb_rows - 1) / rb_rows;
    }
  }
  if (nrb > 1) {
    if (nF == kNT)
      k_col_sums<T, kNT><<<dim3(ns, nrb, G), kNT * 32, 0, s>>>(jobs, rb_rows);
    else
      k_col_sums<T, 12><<<dim3(ns, nrb, G), 12 * 32, 0, s>>>(jobs, rb_rows);
  }
  if (nF == kNT)
    k_sat_tile<T, kNT><<<dim3(ns, nrb, G), kNT * 32, 0, s>>>(jobs, rb_rows);
  else
    k_sat_tile<T, 12><<<dim3(ns, nrb, G), 12 * 32, 0, s>>>(jobs, rb_rows);
  k_query_consts<<<G, kDiagMaxL * kNT, 0, s>>>(jobs, nF);
  const DiagDist none{};
  if (dist) {
    k_query<MT, false, true><<<dim3(qblocks, nL, 2 * G), 256, 0, s>>>(jobs, nF, origins, nullptr,
                                                                       *dist);
  } else {
    const dim3 qg(qblocks, nL, G);
    if (per_box)
      k_query<MT, true, false><<<qg, 256, 0, s>>>(jobs, nF, origins, per_box, none);
    else
      k_query<MT, false, false><<<qg, 256, 0, s>>>(jobs, nF, origins, nullptr, none);
  }
  k_stats_final<MT><<<dim3(nL, G), 384, 0, s>>>(jobs, stats, dist ? dist->mach : nullptr);
  return cudaGetLastError();
}

}  // namespace

cudaError_t diag_moments(const Member &hm, const double *snap3, double *rho, double *ux,
                         double *uy, double *omega, const DiagScratch &sc, cudaStream_t s) {
  const Grid g = grid_of(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  double *U = ux ? ux : sc.f + (size_t)kSnapSlots * N;
  double *V = uy ? uy : sc.f + (size_t)(kSnapSlots + 1) * N;
  dim3 b(32, 8);
  k_moments<<<cells_grid(g, b), b, 0, s>>>(g, snap3, N, rho, U, V);
  if (omega) k_vorticity<<<cells_grid(g, b), b, 0, s>>>(g, U, V, omega);
  return cudaGetLastError();
}

cudaError_t diag_global(const Member &hm, const double *snap3, const DiagScratch &sc,
                        double *out7_dev, cudaStream_t s) {
  Grid g = grid_of(hm);
  const size_t N = (size_t)hm.nx * hm.ny;
  // snap3 holds (rho, j_x, j_y) and, with a variable-viscosity collision,
  // the local viscosity as a fourth field
  if (hm.collision != 0) g.nu_field = snap3 + 3 * N;
  double *U = sc.f + (size_t)(kSnapSlots + 1) * N, *V = sc.f + (size_t)(kSnapSlots + 2) * N;
  dim3 b(32, 8);
  k_moments<<<cells_grid(g, b), b, 0, s>>>(g, snap3, N, nullptr, U, V);
  int nblocks = (int)((N + 255) / 256);
  if (nblocks > kMaxPartialBlocks) nblocks = kMaxPartialBlocks;
  k_global<<<nblocks, dim3(32, 8), 0, s>>>(g, snap3, U, V, N, sc.partials);
  k_sum_partials<<<1, 256, 0, s>>>(sc.partials, nblocks, 7, out7_dev);
  k_global_scale<<<1, 32, 0, s>>>(out7_dev, N);
  return cudaGetLastError();
}

// Box lists: about 8 boxes per thread pair; every periodic origin: about 32
// per thread pair; at most kMaxQueryBlocks CTAs per (job, size, part).  A
// batch of few jobs with few boxes (a small grid) gets smaller CTAs, down to
// one pass of 128 boxes, about 256 per size over the batch: its FP64
// statistics then spread over the SMs instead of queueing on a few (GB300
// issues about 1.7 FP64 FMAs per clock per SM).
int diag_query_blocks(int max_boxes, bool origin_list, int batch_jobs) {
  const int per_cta = origin_list ? 1024 : 4096;
  int qb = (max_boxes + per_cta - 1) / per_cta;
  const int want = (256 + std::max(1, batch_jobs) - 1) / std::max(1, batch_jobs);
  qb = std::max(qb, std::min(want, (max_boxes + 127) / 128));
  return std::min(kMaxQueryBlocks, std::max(1, qb));
}

size_t diag_slot_doubles(size_t Nmax, size_t pad) {
  // snapshot slots + term-stage fields + kNT padded tables, in whole 256-byte
  // units (so field rows keep the 16-byte alignment of vector loads)
  const size_t d = (size_t)(kSnapSlots + NF) * Nmax + kNT * (Nmax + pad);
  return (d + 31) / 32 * 32;
}

size_t diag_job_partials(size_t Nmax, size_t pad) {
  // CTAs of the 32 x 8 cell grid: ceil(nx/32) ceil(ny/8) <= N/256 + pad/8 + 1
  const size_t ctas = Nmax / 256 + pad / 8 + 2;
  return kPartMax + kNT * ctas;  // 8-byte words
}

cudaError_t diag_balance(const DiagJob *jobs_host, const DiagJob *jobs_dev, int G,
                         int precision, bool pairs, const int *origins_dev,
                         double *stats_dev, double *per_box_dev, const DiagDist *dist,
                         cudaStream_t s) {
  if (G < 1 || (per_box_dev && G != 1) || (per_box_dev && dist)) return cudaErrorInvalidValue;
  if (dist && (dist->n_delta < 1 || dist->n_delta > kDiagMaxEdges || dist->n_mach < 1 ||
               dist->n_mach > kDiagMaxEdges))
    return cudaErrorInvalidValue;
  if (precision == 32)
    return balance_launches<float, float>(jobs_host, jobs_dev, G, pairs, origins_dev,
                                          stats_dev, per_box_dev, dist, s);
  return balance_launches<double, double>(jobs_host, jobs_dev, G, pairs, origins_dev,
                                          stats_dev, per_box_dev, dist, s);
}

}  // namespace lbm
