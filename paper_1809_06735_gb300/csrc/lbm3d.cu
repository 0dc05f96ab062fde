// Three-dimensional extension (include/lbm3d.h): D3Q19 and D3Q27 BGK stream-collide
// with exact-difference forcing (eq. (1), eq. (2), Sec. 3 of Tauzin et al.
// 2018) and the sub-volume energy/enstrophy balance of eqs. (8)-(13) in the
// general index forms, with vortex stretching, over L x L x L boxes.
//
// Storage: double buffer, pull layout pop[b][l][z][y][x] (x fastest): the
// pre-collision f_l(x, n) = pop[cur][l][x - c_l].  FP32 stores deviations
// g = f - t rho0, FP64 f.  One thread per cell; one launch per member.
//
// Diagnostic (FP64 arithmetic): snapshots (rho, j_x, j_y, j_z) of the levels
// n, n-1, n-2 (FP32 storage: compensated sums of the FP32 populations, so
// the FP64 value of the stored state); four term passes; 13 exact 64-bit
// fixed-point summed-volume tables (scale 2^e per field with N max|T| 2^e <
// 2^62); 8-corner box sums in modular integer arithmetic; FP64 statistics
// with fixed-order reductions.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lbm3d.h"

namespace {

// Velocity sets: D3Q27 = rest, 6 axis, 12 edge, 8 corner velocities in the
// order of include/lbm3d.h; D3Q19 is its first 19 entries.  Weights by
// |c|^2: D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216.
__host__ __device__ constexpr int c3x(int l) {
  return (l == 1 || l == 7 || l == 9 || l == 11 || l == 13 || l == 19 || l == 21 || l == 23 ||
          l == 26) ? 1
         : (l == 2 || l == 8 || l == 10 || l == 12 || l == 14 || l == 20 || l == 22 || l == 24 ||
            l == 25) ? -1 : 0;
}
__host__ __device__ constexpr int c3y(int l) {
  return (l == 3 || l == 7 || l == 10 || l == 15 || l == 17 || l == 19 || l == 21 || l == 24 ||
          l == 25) ? 1
         : (l == 4 || l == 8 || l == 9 || l == 16 || l == 18 || l == 20 || l == 22 || l == 23 ||
            l == 26) ? -1 : 0;
}
__host__ __device__ constexpr int c3z(int l) {
  return (l == 5 || l == 11 || l == 14 || l == 15 || l == 18 || l == 19 || l == 22 || l == 23 ||
          l == 25) ? 1
         : (l == 6 || l == 12 || l == 13 || l == 16 || l == 17 || l == 20 || l == 21 || l == 24 ||
            l == 26) ? -1 : 0;
}
template <int Q>
__host__ __device__ constexpr double w3(int l) {
  return Q == 27 ? (l == 0 ? 8.0 / 27.0 : (l <= 6 ? 2.0 / 27.0 : (l <= 18 ? 1.0 / 54.0 : 1.0 / 216.0)))
                 : (l == 0 ? 1.0 / 3.0 : (l <= 6 ? 1.0 / 18.0 : 1.0 / 36.0));
}

struct M3 {
  int nx, ny, nz, force_kind, kf, q;  // q: 19 or 27 velocities
  long long item0, items;  // the member's work items of the four-cell kernel (0: not in it)
  double tau, omega, rho0, F0, alpha, nu;
  float rho0_f, omega_f, alpha_f, F0_f;
  size_t N;
  void *pop[2];
  double *snap;  // ring [3 slots][4][N]: rho, jx, jy, jz
  void *ftab;    // force kind 1: F_x(y) [ny], F_y(z) [nz], F_z(x) [nx] (storage precision)
  double *ftab64;  // the same in FP64
};

__device__ __forceinline__ int wrp(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ size_t cell(const M3 &M, int x, int y, int z) {
  return ((size_t)z * M.ny + y) * M.nx + x;
}

// External force of the cyclic Kolmogorov kind at (x, y, z), from the
// per-axis tables (zero tables for force kind 0).
template <typename T>
__device__ __forceinline__ void force3(const M3 &M, const T *tab, int x, int y, int z, T &fx,
                                       T &fy, T &fz) {
  fx = tab[y];
  fy = tab[M.ny + z];
  fz = tab[M.ny + M.nz + x];
}

// BGK + EDM collision of one cell in storage form (FP32: deviations).
template <typename T, int Q>
__device__ __forceinline__ void collide3(T v[Q], T rho0, T om, T Fex, T Fey, T Fez, T alpha) {
  T dr = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    dr += v[l];
    jx += (T)c3x(l) * v[l];
    jy += (T)c3y(l) * v[l];
    jz += (T)c3z(l) * v[l];
  }
  const T rho = sizeof(T) == 4 ? rho0 + dr : dr;
  const T drho = sizeof(T) == 4 ? dr : dr - rho0;  // FP64: rho0 passed as 0
  const T ir = T(1) / rho;
  const T ux = jx * ir, uy = jy * ir, uz = jz * ir;
  const T Fx = Fex - alpha * jx, Fy = Fey - alpha * jy, Fz = Fez - alpha * jz;
  const T dux = Fx * ir, duy = Fy * ir, duz = Fz * ir;
  const T usq = ux * ux + uy * uy + uz * uz;
  const T dsq = dux * (T(2) * ux + dux) + duy * (T(2) * uy + duy) + duz * (T(2) * uz + duz);
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const T t = (T)w3<Q>(l);
    const T cu = (T)c3x(l) * ux + (T)c3y(l) * uy + (T)c3z(l) * uz;
    const T cd = (T)c3x(l) * dux + (T)c3y(l) * duy + (T)c3z(l) * duz;
    T eq;
    if constexpr (sizeof(T) == 4)
      eq = t * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
    else
      eq = t * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
    const T Fl = t * rho * (T(3) * cd + T(4.5) * cd * (T(2) * cu + cd) - T(1.5) * dsq);
    v[l] = v[l] - om * (v[l] - eq) + Fl;
  }
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k3_step(const M3 *__restrict__ ms, int member, int cur) {
  const M3 &M = ms[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y,
            z = blockIdx.z;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(M.pop[cur]);
  T *dst = static_cast<T *>(M.pop[cur ^ 1]);
  const size_t N = M.N;
  T v[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l)
    v[l] = src[(size_t)l * N + cell(M, wrp(x - c3x(l), M.nx), wrp(y - c3y(l), M.ny),
                                    wrp(z - c3z(l), M.nz))];
  T fx, fy, fz;
  force3<T>(M, static_cast<const T *>(M.ftab), x, y, z, fx, fy, fz);
  if constexpr (sizeof(T) == 4)
    collide3<float, Q>(v, M.rho0_f, M.omega_f, fx, fy, fz, M.alpha_f);
  else
    collide3<double, Q>(v, 0.0, M.omega, fx, fy, fz, M.alpha);
  const size_t c = cell(M, x, y, z);
#pragma unroll
  for (int l = 0; l < Q; ++l) dst[(size_t)l * N + c] = v[l];
}

// FP32 stream-collide with CPL = 4 or 2 consecutive cells per lane
// (nx % 4 == 0), all such members in one persistent launch: a work item is 4
// rows (y0 .. y0+3) of a 32 CPL-cell x segment of one z plane of one member,
// a warp per row; the items of every member are numbered consecutively
// (M3::item0, M3::items).  Each population is one aligned 16- or 8-byte load
// per lane from its source row (y - c_y, z - c_z); the -+1 x-shift is a
// warp shuffle with one scalar load at the segment's edges (the periodic
// wrap included), as in 2D.  Two cells per lane halve the registers that
// hold the pulled populations (2 Q instead of 4 Q), for more resident warps.
template <int CPL>
struct Vec3;
template <>
struct Vec3<4> {
  using V = float4;
  static __device__ __forceinline__ float first(const V &o) { return o.x; }
  static __device__ __forceinline__ float lastv(const V &o) { return o.w; }
  static __device__ __forceinline__ void get(const V &o, float *v) {
    v[0] = o.x; v[1] = o.y; v[2] = o.z; v[3] = o.w;
  }
  static __device__ __forceinline__ V make(const float *v) { return make_float4(v[0], v[1], v[2], v[3]); }
  static __device__ __forceinline__ V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct Vec3<2> {
  using V = float2;
  static __device__ __forceinline__ float first(const V &o) { return o.x; }
  static __device__ __forceinline__ float lastv(const V &o) { return o.y; }
  static __device__ __forceinline__ void get(const V &o, float *v) { v[0] = o.x; v[1] = o.y; }
  static __device__ __forceinline__ V make(const float *v) { return make_float2(v[0], v[1]); }
  static __device__ __forceinline__ V zero() { return make_float2(0.f, 0.f); }
};

template <int Q, int CPL>
__global__ void __launch_bounds__(128, CPL == 2 ? (Q == 19 ? 5 : 4) : (Q == 19 ? 4 : 3))
    k3_step_vec(const M3 *__restrict__ ms, int n_members, long long n_items, int cur, int flip) {
  using VT = Vec3<CPL>;
  using V = typename VT::V;
  constexpr int SEG = 32 * CPL;
  const int lane = threadIdx.x;
  // the current member's parameters, reloaded only when the items move on
  // to another member; flip walks the items in reverse order, so that a step
  // starts where the previous one ended (those populations are still in L2)
  int m = -1, nx = 0, ny = 0, nz = 0;
  long long item0 = 0, item1 = 0;
  size_t N = 0;
  const float *src = nullptr, *tab = nullptr;
  float *dst = nullptr;
  float rho0 = 0.f, om = 0.f, alpha = 0.f;
  for (long long t = blockIdx.x; t < n_items; t += gridDim.x) {
    const long long it = flip ? n_items - 1 - t : t;
    if (it < item0 || it >= item1) {
      m = 0;
      while (m + 1 < n_members && it >= ms[m].item0 + ms[m].items) ++m;
      const M3 &M = ms[m];
      nx = M.nx;
      ny = M.ny;
      nz = M.nz;
      item0 = M.item0;
      item1 = M.item0 + M.items;
      N = M.N;
      src = static_cast<const float *>(M.pop[cur]);
      dst = static_cast<float *>(M.pop[cur ^ 1]);
      tab = static_cast<const float *>(M.ftab);
      rho0 = M.rho0_f;
      om = M.omega_f;
      alpha = M.alpha_f;
    }
    const unsigned li = (unsigned)(it - item0);  // < 2^28 items per member
    const unsigned gx = (unsigned)(nx + SEG - 1) / (unsigned)SEG, gy = (unsigned)(ny + 3) / 4u;
    const unsigned lx = li / gx;
    const int xs = (int)(li - lx * gx), yg = (int)(lx % gy), z = (int)(lx / gy);
    const int x = xs * SEG + CPL * lane, y = yg * 4 + threadIdx.y;
    if (y >= ny) continue;  // whole warps
    const bool active = x < nx;
    const bool last = active && (lane == 31 || x + CPL >= nx);
    const int xprev = x == 0 ? nx - 1 : x - 1, xnext = x + CPL >= nx ? 0 : x + CPL;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y + 1 == ny ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z + 1 == nz ? 0 : z + 1;
    const size_t rowy[3] = {(size_t)yp * nx, (size_t)y * nx, (size_t)ym * nx};
    const size_t slab[3] = {(size_t)zp * ny * nx, (size_t)z * ny * nx, (size_t)zm * ny * nx};
    float v[Q][CPL];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      // pull from (y - c_y, z - c_z): entry 1 + c of the (+1, 0, -1) neighbours
      const float *row = src + (size_t)l * N + slab[1 + c3z(l)] + rowy[1 + c3y(l)];
      V o = VT::zero();
      if (active) o = __ldg(reinterpret_cast<const V *>(row + x));
      float a[CPL];
      VT::get(o, a);
      if (c3x(l) == 0) {
#pragma unroll
        for (int i = 0; i < CPL; ++i) v[l][i] = a[i];
      } else if (c3x(l) > 0) {  // from x - 1
        float prev = __shfl_up_sync(0xffffffffu, VT::lastv(o), 1);
        if (active && (lane == 0 || x == 0)) prev = __ldg(row + xprev);
        v[l][0] = prev;
#pragma unroll
        for (int i = 1; i < CPL; ++i) v[l][i] = a[i - 1];
      } else {  // from x + 1
        float next = __shfl_down_sync(0xffffffffu, VT::first(o), 1);
        if (last) next = __ldg(row + xnext);
#pragma unroll
        for (int i = 0; i + 1 < CPL; ++i) v[l][i] = a[i + 1];
        v[l][CPL - 1] = next;
      }
    }
    if (!active) continue;
    const float fx = tab[y], fy = tab[ny + z];
    const size_t c = slab[1] + rowy[1] + x;
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
      float g[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) g[l] = v[l][i];
      collide3<float, Q>(g, rho0, om, fx, fy, tab[ny + nz + x + i], alpha);
#pragma unroll
      for (int l = 0; l < Q; ++l) v[l][i] = g[l];
    }
#pragma unroll
    for (int l = 0; l < Q; ++l)
      __stcs(reinterpret_cast<V *>(dst + (size_t)l * N + c), VT::make(v[l]));
  }
}

template <typename T, int Q>
__global__ void k3_init(const M3 *__restrict__ ms, int member, int cur, const double *rho,
                        const double *ux, const double *uy, const double *uz) {
  const M3 &M = ms[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y,
            z = blockIdx.z;
  if (x >= M.nx || y >= M.ny) return;
  const size_t c = cell(M, x, y, z);
  const double r = rho[c], u = ux[c], v = uy[c], w = uz[c], uu = u * u + v * v + w * w;
  T *dst = static_cast<T *>(M.pop[cur]);
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const double cu = c3x(l) * u + c3y(l) * v + c3z(l) * w;
    const double feq = w3<Q>(l) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    // the population at x is stored at its pull origin x - c_l
    const size_t o = cell(M, wrp(x - c3x(l), M.nx), wrp(y - c3y(l), M.ny), wrp(z - c3z(l), M.nz));
    dst[(size_t)l * M.N + o] = (T)(sizeof(T) == 4 ? feq - w3<Q>(l) * M.rho0 : feq);
  }
}

// Public <-> storage (to_public: storage -> f[19][N] doubles).
template <typename T, int Q>
__global__ void k3_copy(const M3 *__restrict__ ms, int member, int cur, double *f, int to_public) {
  const M3 &M = ms[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y,
            z = blockIdx.z;
  if (x >= M.nx || y >= M.ny) return;
  const size_t c = cell(M, x, y, z);
  T *st = static_cast<T *>(M.pop[cur]);
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const size_t o = (size_t)l * M.N +
                     cell(M, wrp(x - c3x(l), M.nx), wrp(y - c3y(l), M.ny), wrp(z - c3z(l), M.nz));
    const double off = sizeof(T) == 4 ? w3<Q>(l) * M.rho0 : 0.0;
    if (to_public)
      f[(size_t)l * M.N + c] = (double)st[o] + off;
    else
      st[o] = (T)(f[(size_t)l * M.N + c] - off);
  }
}

__device__ __forceinline__ void two_sum3(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (rho, j) of the current state into snapshot slot `slot` (FP64; FP32
// storage by compensated FP32 sums of the stored deviations).
template <typename T, int Q>
__global__ void k3_snapshot(const M3 *__restrict__ ms, int member, int cur, int slot) {
  const M3 &M = ms[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y,
            z = blockIdx.z;
  if (x >= M.nx || y >= M.ny) return;
  const T *st = static_cast<const T *>(M.pop[cur]);
  T v[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l)
    v[l] = st[(size_t)l * M.N + cell(M, wrp(x - c3x(l), M.nx), wrp(y - c3y(l), M.ny),
                                     wrp(z - c3z(l), M.nz))];
  double out[4];
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float s = 0.f, e = 0.f;
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        const int c = q == 0 ? 1 : (q == 1 ? c3x(l) : (q == 2 ? c3y(l) : c3z(l)));
        if (c == 0) continue;
        float d;
        two_sum3(s, c > 0 ? v[l] : -v[l], s, d);
        e += d;
      }
      out[q] = (double)s + (double)e;
    }
    out[0] += M.rho0;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = 0.0;
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      out[0] += v[l];
      out[1] += c3x(l) * v[l];
      out[2] += c3y(l) * v[l];
      out[3] += c3z(l) * v[l];
    }
  }
  double *d = M.snap + (size_t)slot * 4 * M.N;
  const size_t c = cell(M, x, y, z);
#pragma unroll
  for (int q = 0; q < 4; ++q) d[(size_t)q * M.N + c] = out[q];
}

// ---------------------------------------------------------------------------
// Diagnostic (FP64)
// ---------------------------------------------------------------------------

// scratch field indices (each N doubles)
enum F3 {
  UX0, UY0, UZ0, DU01X, DU01Y, DU01Z, DU12X, DU12Y, DU12Z, R0, DR, FRX, FRY, FRZ, WX, WY, WZ,
  EUX, EUY, EUZ, CUX, CUY, CUZ, OUX, OUY, OUZ, SXX, SXY, SXZ, SYY, SYZ, SZZ, HWX, HWY, HWZ,
  T3,  // T3 .. T3 + 12: the 13 term fields
  NF3 = T3 + 13
};

struct Diag3 {
  const M3 *m;
  const double *s0, *s1, *s2;  // snapshots of n, n-1, n-2
  double *f;                   // NF3 fields of N doubles, then the tables
};

// Periodic index for i in [-4, n + 4): one compare for n >= 4, a modulo for
// the tiny grids.
__device__ __forceinline__ int wrap4(int i, int n) {
  if (n >= 4) return i < 0 ? i + n : (i >= n ? i - n : i);
  return ((i % n) + n) % n;
}

// Eq. (18) along axis a (0 x, 1 y, 2 z), periodic, in the arithmetic type T.
template <typename T>
__device__ __forceinline__ T D3(const M3 &M, const T *A, int x, int y, int z, int a) {
  const T cf[4] = {T(0.8), T(-0.2), T(4.0 / 105.0), T(-1.0 / 280.0)};
  T s = T(0);
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    size_t p, q;
    if (a == 0) {
      p = cell(M, wrap4(x + k, M.nx), y, z);
      q = cell(M, wrap4(x - k, M.nx), y, z);
    } else if (a == 1) {
      p = cell(M, x, wrap4(y + k, M.ny), z);
      q = cell(M, x, wrap4(y - k, M.ny), z);
    } else {
      p = cell(M, x, y, wrap4(z + k, M.nz));
      q = cell(M, x, y, wrap4(z - k, M.nz));
    }
    s += cf[k - 1] * (A[p] - A[q]);
  }
  return s;
}

// One thread per cell; scratch field k holds N values of T in its N-double
// slot.
#define D3CELL                                                                   \
  const M3 &M = *J.m;                                                            \
  const int x = blockIdx.x * blockDim.x + threadIdx.x,                           \
            y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;           \
  if (x >= M.nx || y >= M.ny) return;                                            \
  const size_t N = M.N, c = cell(M, x, y, z);                                    \
  auto F = [&](int k) { return reinterpret_cast<T *>(J.f + (size_t)k * N); };

// Pass 0.  Bare momentum j and u = (j + F/2)/rho with F = F_ext - alpha j,
// i.e. rho u = m = (1 - alpha/2) j + F_ext/2.  The level differences of rho
// and j are formed in FP64 from the FP64 snapshots and rounded once to T;
// u^n - u^{n-1} = ((1 - alpha/2)(j^n - j^{n-1}) - u^n (rho^n - rho^{n-1}))
// / rho^{n-1} (exact identity), and E^n - E^{n-1} = [drho |u^n|^2 +
// rho^{n-1} du . (2 u^n - du)] / 2, so LHS^E = (3 dE01 - dE12)/2 (eq. 17)
// carries no cancellation of the level values themselves.  Stores u^n, the
// two velocity differences, rho, rho - rho0, F/rho; LHS^E and
// RHS^{E,3} = u . F.
template <typename T>
__global__ void k3_prep(Diag3 J) {
  D3CELL;
  double fxd, fyd, fzd;
  force3<double>(M, M.ftab64, x, y, z, fxd, fyd, fzd);
  const double *S0 = J.s0, *S1 = J.s1, *S2 = J.s2;
  const double r0d = S0[c], r1d = S1[c], r2d = S2[c];
  T j0[3], dj01[3], dj12[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const size_t o = (size_t)(i + 1) * N + c;
    j0[i] = (T)S0[o];
    dj01[i] = (T)(S0[o] - S1[o]);
    dj12[i] = (T)(S1[o] - S2[o]);
  }
  const T r0 = (T)r0d, r1 = (T)r1d, r2 = (T)r2d;
  const T dr01 = (T)(r0d - r1d), dr12 = (T)(r1d - r2d);
  const T a = (T)M.alpha, ca = T(1) - T(0.5) * a;
  const T fe[3] = {(T)fxd, (T)fyd, (T)fzd};
  T u0[3], du01[3], du12[3], Fv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Fv[i] = fe[i] - a * j0[i];
    u0[i] = (j0[i] + T(0.5) * Fv[i]) / r0;
  }
  T q0 = T(0), q1 = T(0), p01 = T(0), p12 = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    du01[i] = (ca * dj01[i] - u0[i] * dr01) / r1;
    const T u1 = u0[i] - du01[i];
    du12[i] = (ca * dj12[i] - u1 * dr12) / r2;
    q0 += u0[i] * u0[i];
    q1 += u1 * u1;
    p01 += du01[i] * (T(2) * u0[i] - du01[i]);
    p12 += du12[i] * (T(2) * u1 - du12[i]);
  }
  const T dE01 = T(0.5) * (dr01 * q0 + r1 * p01);
  const T dE12 = T(0.5) * (dr12 * q1 + r2 * p12);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    F(UX0 + i)[c] = u0[i];
    F(DU01X + i)[c] = du01[i];
    F(DU12X + i)[c] = du12[i];
    F(FRX + i)[c] = Fv[i] / r0;
  }
  F(R0)[c] = r0;
  F(DR)[c] = (T)(r0d - M.rho0);
  F(T3 + 0)[c] = T(0.5) * (T(3) * dE01 - dE12);
  F(T3 + 3)[c] = u0[0] * Fv[0] + u0[1] * Fv[1] + u0[2] * Fv[2];
}

// Pass 1: velocity gradients G_ij = d_j u_i at n, the vorticity w^n and its
// level differences dw = curl(du) (LHS^Omega = (3 dO01 - dO12)/2 with
// O^n - O^{n-1} = dw01 . (2 w^n - dw01)/2), S, RHS^{E,2}, RHS^{E,4},
// RHS^{O,2}, RHS^{O,3}, RHS^{O,6}, and the fluxes of pass 2.
template <typename T>
__global__ void k3_grad(Diag3 J) {
  D3CELL;
  T G[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[i][j] = D3<T>(M, F(UX0 + i), x, y, z, j);
  T w0[3];
  w0[0] = G[2][1] - G[1][2];
  w0[1] = G[0][2] - G[2][0];
  w0[2] = G[1][0] - G[0][1];
  T dO[2];
  T w1[3];
  for (int m = 0; m < 2; ++m) {
    const T *U = F((m ? DU12X : DU01X)), *V = F((m ? DU12Y : DU01Y)), *W = F((m ? DU12Z : DU01Z));
    const T dw[3] = {D3<T>(M, W, x, y, z, 1) - D3<T>(M, V, x, y, z, 2),
                     D3<T>(M, U, x, y, z, 2) - D3<T>(M, W, x, y, z, 0),
                     D3<T>(M, V, x, y, z, 0) - D3<T>(M, U, x, y, z, 1)};
    const T *wl = m ? w1 : w0;  // the later level of the pair
    T p = T(0);
    for (int i = 0; i < 3; ++i) p += dw[i] * (T(2) * wl[i] - dw[i]);
    dO[m] = T(0.5) * p;
    if (m == 0)
      for (int i = 0; i < 3; ++i) w1[i] = w0[i] - dw[i];
  }
  F(T3 + 6)[c] = T(0.5) * (T(3) * dO[0] - dO[1]);
  const T Om0 = T(0.5) * (w0[0] * w0[0] + w0[1] * w0[1] + w0[2] * w0[2]);
  const T u[3] = {F(UX0)[c], F(UY0)[c], F(UZ0)[c]}, r = F(R0)[c];
  const T nr = (T)M.nu * r;
  T S[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = G[i][j] + G[j][i];
  T gp = T(0), sd = T(0), st = T(0);
  for (int i = 0; i < 3; ++i) gp += u[i] * D3<T>(M, F(DR), x, y, z, i) / T(3);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      sd += S[i][j] * G[i][j];
      st += w0[i] * w0[j] * G[i][j];
    }
  const T div = G[0][0] + G[1][1] + G[2][2];
  T cf = T(0);  // omega . curl(F / rho)
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    cf += w0[i] * (D3<T>(M, F(FRX + k), x, y, z, j) - D3<T>(M, F(FRX + j), x, y, z, k));
  }
  F(T3 + 2)[c] = -gp;
  F(T3 + 4)[c] = -nr * sd;
  F(T3 + 8)[c] = -Om0 * div;
  F(T3 + 9)[c] = cf;
  F(T3 + 12)[c] = st;
  const T E0 = T(0.5) * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  for (int j = 0; j < 3; ++j) {
    F(EUX + j)[c] = E0 * u[j];
    F(OUX + j)[c] = Om0 * u[j];
    F(CUX + j)[c] = nr * (u[0] * S[0][j] + u[1] * S[1][j] + u[2] * S[2][j]);
    F(WX + j)[c] = w0[j];
  }
  F(SXX)[c] = nr * S[0][0];
  F(SXY)[c] = nr * S[0][1];
  F(SXZ)[c] = nr * S[0][2];
  F(SYY)[c] = nr * S[1][1];
  F(SYZ)[c] = nr * S[1][2];
  F(SZZ)[c] = nr * S[2][2];
}

// Pass 2: RHS^{E,1}, RHS^{E,5}, RHS^{O,1}; H_i = d_j(nu rho S_ij)/rho;
// RHS^{O,4} = H . curl(omega); H x omega for pass 3.
template <typename T>
__global__ void k3_flux(Diag3 J) {
  D3CELL;
  T e1 = T(0), e5 = T(0), o1 = T(0);
  for (int j = 0; j < 3; ++j) {
    e1 -= D3<T>(M, F(EUX + j), x, y, z, j);
    e5 += D3<T>(M, F(CUX + j), x, y, z, j);
    o1 -= D3<T>(M, F(OUX + j), x, y, z, j);
  }
  const int sidx[3][3] = {{SXX, SXY, SXZ}, {SXY, SYY, SYZ}, {SXZ, SYZ, SZZ}};
  const T r = F(R0)[c];
  T H[3];
  for (int i = 0; i < 3; ++i) {
    T h = T(0);
    for (int j = 0; j < 3; ++j) h += D3<T>(M, F(sidx[i][j]), x, y, z, j);
    H[i] = h / r;
  }
  T o4 = T(0);
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    o4 += H[i] * (D3<T>(M, F(WX + k), x, y, z, j) - D3<T>(M, F(WX + j), x, y, z, k));
  }
  const T w[3] = {F(WX)[c], F(WY)[c], F(WZ)[c]};
  F(T3 + 1)[c] = e1;
  F(T3 + 5)[c] = e5;
  F(T3 + 7)[c] = o1;
  F(T3 + 10)[c] = o4;
  for (int j = 0; j < 3; ++j) {
    const int a = (j + 1) % 3, b = (j + 2) % 3;
    F(HWX + j)[c] = H[a] * w[b] - H[b] * w[a];
  }
}

// Pass 3: RHS^{O,5} = div(H x omega).
template <typename T>
__global__ void k3_curl(Diag3 J) {
  D3CELL;
  T s = T(0);
  for (int j = 0; j < 3; ++j) s += D3<T>(M, F(HWX + j), x, y, z, j);
  F(T3 + 11)[c] = s;
}

// Summed-volume tables: table k at tab + k * (nx+1)(ny+1)(nz+1), exclusive
// prefix P(x, y, z) over x' < x, y' < y, z' < z (the zero planes included).
__device__ __forceinline__ size_t tidx(const M3 &M, int x, int y, int z) {
  return ((size_t)z * (M.ny + 1) + y) * (M.nx + 1) + x;
}

// Largest |T_k| per term field: grid (CTAs, 13), each CTA a strided share
// of the cells, combined with an integer atomicMax on the bit pattern
// (non-negative doubles order like their bits; NaN counts as 0).  maxbits
// [13] must be zero on entry.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  return b <= 0x7ff0000000000000ull ? b : 0ull;
}
__device__ __forceinline__ unsigned long long abs_bits(float v) {  // as the double's bits
  const float a = fabsf(v);
  return a == a ? (unsigned long long)__double_as_longlong((double)a) : 0ull;
}

template <typename T>
__global__ void __launch_bounds__(256) k3_absmax(Diag3 J, unsigned long long *maxbits) {
  const M3 &M = *J.m;
  const int k = blockIdx.y;
  const T *A = reinterpret_cast<const T *>(J.f + (size_t)(T3 + k) * M.N);
  unsigned long long m = 0ull;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M.N;
       i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long b = abs_bits(A[i]);
    if (b > m) m = b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long n = __shfl_xor_sync(0xffffffffu, m, o);
    m = n > m ? n : m;
  }
  __shared__ unsigned long long sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = sh[w] > m ? sh[w] : m;
    atomicMax(maxbits + k, m);
  }
}

// Scales 2^e with N max |T_k| 2^e < 2^62 (every partial sum fits int64):
// maxes[k] = 2^e, maxes[16 + k] = e, maxes[80 + k] = 2^-e (one thread per field).
__global__ void k3_scales(Diag3 J, const unsigned long long *maxbits, double *maxes) {
  const M3 &M = *J.m;
  const int k = threadIdx.x;
  if (k >= 13) return;
  const double mx = __longlong_as_double((long long)maxbits[k]);
  int e = 0;
  if (mx > 0.0) {
    int ex, nbits = 0;
    frexp(mx, &ex);  // mx < 2^ex
    while (((size_t)1 << nbits) < M.N) ++nbits;
    e = 62 - nbits - ex;
    if (e > 1000) e = 1000;
  }
  maxes[k] = ldexp(1.0, e);
  maxes[16 + k] = (double)e;
  maxes[80 + k] = ldexp(1.0, -e);
}

// Quantised values scanned along x: one thread per (y, z, field) row.
template <typename T>
__global__ void k3_scan_x(Diag3 J, const double *scales, long long *tab) {
  const M3 &M = *J.m;
  const int y = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y, k = blockIdx.z;
  if (y > M.ny || z > M.nz) return;
  const size_t ts = (size_t)(M.nx + 1) * (M.ny + 1) * (M.nz + 1);
  long long *t = tab + (size_t)k * ts;
  if (y == 0 || z == 0) {  // zero planes
    for (int x = 0; x <= M.nx; ++x) t[tidx(M, x, y, z)] = 0;
    return;
  }
  const T *A = reinterpret_cast<const T *>(J.f + (size_t)(T3 + k) * M.N);
  const double sc = scales[k];
  long long acc = 0;
  t[tidx(M, 0, y, z)] = 0;
  for (int x = 0; x < M.nx; ++x) {
    acc += __double2ll_rn((double)A[cell(M, x, y - 1, z - 1)] * sc);
    t[tidx(M, x + 1, y, z)] = acc;
  }
}

// Prefix along y (axis 1) or z (axis 2) of the tables in place: one thread
// per (x, other coordinate, field) line.
__global__ void k3_scan_yz(Diag3 J, long long *tab, int axis) {
  const M3 &M = *J.m;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, o = blockIdx.y, k = blockIdx.z;
  if (x > M.nx) return;
  const int no = axis == 1 ? M.nz : M.ny, nl = axis == 1 ? M.ny : M.nz;
  if (o > no) return;
  const size_t ts = (size_t)(M.nx + 1) * (M.ny + 1) * (M.nz + 1);
  long long *t = tab + (size_t)k * ts;
  long long acc = 0;
  for (int i = 1; i <= nl; ++i) {
    const size_t p = axis == 1 ? tidx(M, x, i, o) : tidx(M, x, o, i);
    acc += t[p];
    t[p] = acc;
  }
}

// Exclusive prefix at (x, y, z) for 0 <= x < 2 nx etc. (periodic extension),
// modular arithmetic.
__device__ __forceinline__ unsigned long long P3(const M3 &M, const long long *t, int x, int y,
                                                 int z) {
  unsigned long long v = 0;
  const int qx = x > M.nx, qy = y > M.ny, qz = z > M.nz;
  const int xm = x - qx * M.nx, ym = y - qy * M.ny, zm = z - qz * M.nz;
  for (int a = 0; a <= qx; ++a)
    for (int b = 0; b <= qy; ++b)
      for (int d = 0; d <= qz; ++d)
        v += (unsigned long long)t[tidx(M, a ? M.nx : xm, b ? M.ny : ym, d ? M.nz : zm)];
  return v;
}

template <int NRHS, typename MT>
__device__ __forceinline__ MT delta3(const MT *v) {
  MT sum = MT(0), mx = MT(0);
#pragma unroll
  for (int i = 1; i <= NRHS; ++i) {
    sum += v[i];
    mx = fmax(mx, fabs(v[i]));
  }
  const MT num = fabs(sum - v[0]);
  if (mx == MT(0)) return num == MT(0) ? MT(0) : MT(INFINITY);
  return num / mx;
}

// 64-bit integer to the query precision; the float version assembles the
// IEEE bits with integer instructions (round to nearest, ties away), since
// GB300 runs integer-to-float conversions on its slow FP64 pipe.
template <typename MT>
__device__ __forceinline__ MT i64_to(long long v);
template <>
__device__ __forceinline__ double i64_to<double>(long long v) {
  return (double)v;
}
template <>
__device__ __forceinline__ float i64_to<float>(long long v) {
  const unsigned long long sg = (unsigned long long)v >> 63;
  const unsigned long long a = sg ? 0ull - (unsigned long long)v : (unsigned long long)v;
  if (a == 0ull) return 0.0f;
  int e = 63 - __clzll((long long)a);
  unsigned long long m;
  if (e <= 23) {
    m = a << (23 - e);
  } else {
    const int sh = e - 23;
    m = (a + (1ull << (sh - 1))) >> sh;
    if (m >> 24) {
      m >>= 1;
      ++e;
    }
  }
  return __uint_as_float(((unsigned)sg << 31) | ((unsigned)(e + 127) << 23) |
                         ((unsigned)m & 0x7fffffu));
}

constexpr int kQS3 = 30;  // per size: sums and sums of squares of 15 quantities

// One thread per box: the 13 box sums exactly in integers, their deviations
// from the field means formed in integers too (the mean box sum L^3 total/N,
// rounded) and only then converted to the query precision MT; box means,
// delta^E, delta^Omega; CTA partial sums (fixed order) of the 15 quantities'
// deviations and squares, MT within each warp and FP64 across warps.
template <typename MT>
__global__ void __launch_bounds__(256) k3_query(Diag3 J, const long long *tab,
                                                const double *scales, const double *means,
                                                int L, int nb, const int *origins,
                                                double *partials, double *per_box) {
  const M3 &M = *J.m;
  const size_t ts = (size_t)(M.nx + 1) * (M.ny + 1) * (M.nz + 1);
  __shared__ long long smq[13];
  __shared__ MT scoef[13], smean[13];
  if (threadIdx.x < 13) {
    const int k = threadIdx.x;
    const double vol = (double)L * L * L;
    const long long total = tab[(size_t)k * ts + tidx(M, M.nx, M.ny, M.nz)];
    smq[k] = __double2ll_rn((double)total * (vol / (double)M.N));
    scoef[k] = (MT)(scales[80 + k] / vol);  // 2^-e / L^3
    smean[k] = (MT)means[k];
  }
  __syncthreads();
  MT acc[kQS3];
#pragma unroll
  for (int q = 0; q < kQS3; ++q) acc[q] = MT(0);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    int x0, y0, z0;
    if (origins) {
      x0 = origins[3 * b];
      y0 = origins[3 * b + 1];
      z0 = origins[3 * b + 2];
    } else {
      x0 = b % M.nx;
      y0 = (b / M.nx) % M.ny;
      z0 = b / (M.nx * M.ny);
    }
    MT v[15], d[15];
#pragma unroll 1
    for (int k = 0; k < 13; ++k) {
      const long long *t = tab + (size_t)k * ts;
      const int X0 = x0, X1 = x0 + L, Y0 = y0, Y1 = y0 + L, Z0 = z0, Z1 = z0 + L;
      const unsigned long long s =
          P3(M, t, X1, Y1, Z1) - P3(M, t, X0, Y1, Z1) - P3(M, t, X1, Y0, Z1) - P3(M, t, X1, Y1, Z0) +
          P3(M, t, X0, Y0, Z1) + P3(M, t, X0, Y1, Z0) + P3(M, t, X1, Y0, Z0) - P3(M, t, X0, Y0, Z0);
      d[2 + k] = i64_to<MT>((long long)(s - (unsigned long long)smq[k])) * scoef[k];
      v[2 + k] = d[2 + k] + smean[k];
    }
    v[0] = d[0] = delta3<5>(v + 2);
    v[1] = d[1] = delta3<6>(v + 8);
    if (per_box)
#pragma unroll
      for (int q = 0; q < 15; ++q) per_box[(size_t)b * 15 + q] = (double)v[q];
#pragma unroll
    for (int q = 0; q < 15; ++q) {
      acc[2 * q] += d[q];
      acc[2 * q + 1] += d[q] * d[q];
    }
  }
  __shared__ double sh[kQS3][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kQS3; ++q) {
    MT a = acc[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = (double)a;
  }
  __syncthreads();
  if (threadIdx.x < kQS3) {
    double a = 0.0;
    for (int w = 0; w < 8; ++w) a += sh[threadIdx.x][w];
    partials[(size_t)blockIdx.x * kQS3 + threadIdx.x] = a;
  }
}

// Field means (exact table totals) for the deviation sums of the query.
__global__ void k3_means(Diag3 J, const long long *tab, const double *scales, double *means) {
  const M3 &M = *J.m;
  const int k = threadIdx.x;
  if (k >= 13) return;
  const size_t ts = (size_t)(M.nx + 1) * (M.ny + 1) * (M.nz + 1);
  means[k] = (double)tab[(size_t)k * ts + tidx(M, M.nx, M.ny, M.nz)] / scales[k] / (double)M.N;
}

// Mean and population standard deviation of the 15 quantities of one size
// from the query's CTA partials: a warp per quantity (15 x 32 threads), each
// lane a fixed-order chain over the CTAs, then a shuffle tree.
__global__ void k3_stats(const double *partials, int nblocks, const double *means, int nb,
                         double *stats) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= 15) return;
  double s1 = 0.0, s2 = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    s1 += partials[(size_t)b * kQS3 + 2 * q];
    s2 += partials[(size_t)b * kQS3 + 2 * q + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    const double m1 = s1 / nb;
    stats[2 * q] = (q < 2 ? 0.0 : means[q - 2]) + m1;
    stats[2 * q + 1] = sqrt(fmax(s2 / nb - m1 * m1, 0.0));
  }
}

}  // namespace

struct lbm3d_handle {
  lbm3d_config cfg;
  std::vector<lbm3d_member_cfg> mcfg;
  std::vector<M3> hm;
  M3 *d_m = nullptr;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  int precision = 32;
  int q = 19;  // lattice velocities
  int diag_prec = 64;  // arithmetic of the balance terms
  long long vec_items = 0;  // work items of the vectorised FP32 kernel
  int vec_grid = 0;         // its persistent grid
  int cpl = 4;              // its cells per lane (4 or 2, timed at create)
  cudaStream_t stream = nullptr;
  int cur = 0;
  long long t = 0;
  long long ring_time[3] = {-1, -1, -1};
  double *diag = nullptr;  // NF3 fields + tables + partials, largest member
  size_t diag_doubles = 0;
  int *d_origins = nullptr;
  size_t origin_cap = 0;
  std::string err = "no error";
};

namespace {

thread_local std::string g_err3 = "no error";

int fail3(lbm3d_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  g_err3 = msg;
  return code;
}

// Work items of the vectorised kernel at `cpl` cells per lane (M3::item0,
// M3::items of every FP32 member with nx % 4 == 0), its persistent grid
// (resident CTAs per SM x SMs), and the member table on the device.
cudaError_t vec_layout(lbm3d_handle *h, int cpl) {
  const int seg = 32 * cpl;
  h->vec_items = 0;
  for (size_t m = 0; m < h->hm.size(); ++m) {
    M3 &M = h->hm[m];
    const lbm3d_member_cfg &c = h->mcfg[m];
    M.item0 = h->vec_items;
    M.items = h->precision == 32 && c.nx % 4 == 0
                  ? (long long)((c.nx + seg - 1) / seg) * ((c.ny + 3) / 4) * c.nz : 0;
    h->vec_items += M.items;
  }
  h->cpl = cpl;
  h->vec_grid = 0;
  if (h->vec_items > 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
      const void *k = h->q == 27 ? (cpl == 2 ? (const void *)k3_step_vec<27, 2> : (const void *)k3_step_vec<27, 4>)
                                 : (cpl == 2 ? (const void *)k3_step_vec<19, 2> : (const void *)k3_step_vec<19, 4>);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, 0);
    }
    if (e != cudaSuccess) return e;
    const long long g = (long long)std::max(1, sms) * std::max(1, per_sm);
    h->vec_grid = (int)std::min<long long>(g, h->vec_items);
  }
  return cudaMemcpyAsync(h->d_m, h->hm.data(), sizeof(M3) * h->hm.size(), cudaMemcpyHostToDevice,
                         h->stream);
}

// One step of the vectorised kernel's members.
void launch_vec3(lbm3d_handle *h, cudaStream_t s) {
  const int n = (int)h->mcfg.size();
  const dim3 b(32, 4);
  const int flip = h->cur & 1;
  if (h->q == 27) {
    if (h->cpl == 2)
      k3_step_vec<27, 2><<<h->vec_grid, b, 0, s>>>(h->d_m, n, h->vec_items, h->cur, flip);
    else
      k3_step_vec<27, 4><<<h->vec_grid, b, 0, s>>>(h->d_m, n, h->vec_items, h->cur, flip);
  } else {
    if (h->cpl == 2)
      k3_step_vec<19, 2><<<h->vec_grid, b, 0, s>>>(h->d_m, n, h->vec_items, h->cur, flip);
    else
      k3_step_vec<19, 4><<<h->vec_grid, b, 0, s>>>(h->d_m, n, h->vec_items, h->cur, flip);
  }
}

// The faster of four and two cells per lane on this handle's members: each
// timed over 2 + 4 steps on the live (zeroed) buffers, which are zeroed
// again afterwards (FP32 ensembles above 1 M cells; smaller ones keep 4).
cudaError_t tune_vec3(lbm3d_handle *h) {
  long long cells = 0;
  for (auto &c : h->mcfg) cells += (long long)c.nx * c.ny * c.nz;
  if (h->vec_items == 0 || cells < (1LL << 20)) return cudaSuccess;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  int best_cpl = 4;
  for (int cpl : {4, 2}) {
    if (e == cudaSuccess) e = vec_layout(h, cpl);
    for (int r = 0; r < 6 && e == cudaSuccess; ++r) {
      if (r == 2) e = cudaEventRecord(e0, h->stream);
      launch_vec3(h, h->stream);
      h->cur ^= 1;
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      best_cpl = cpl;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) e = vec_layout(h, best_cpl);
  h->cur = 0;
  const size_t es = h->precision == 32 ? 4 : 8;
  for (size_t m = 0; m < h->hm.size() && e == cudaSuccess; ++m) {
    e = cudaMemsetAsync(h->hm[m].pop[0], 0, es * h->q * h->hm[m].N, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->hm[m].pop[1], 0, es * h->q * h->hm[m].N, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e;
}

#define CK3(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail3(h, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t kAl = 256;
size_t al(size_t v) { return (v + kAl - 1) / kAl * kAl; }
constexpr int kMaxQBlocks3 = 1024;

struct Layout3 {
  size_t members;
  std::vector<size_t> pop0, pop1, snap, ftab, ftab64;
  size_t diag, origins, total, diag_doubles, origin_cap;
};

int lattice_q(const lbm3d_config *cfg) { return cfg->lattice == 27 ? 27 : 19; }

// Launches kernel template K<T, Q> for the handle's precision and lattice.
#define DISPATCH3(h, K, grid, block, ...)                                                   \
  do {                                                                                   \
    if ((h)->precision == 32) {                                                          \
      if ((h)->q == 27) K<float, 27><<<grid, block, 0, (h)->stream>>>(__VA_ARGS__);      \
      else K<float, 19><<<grid, block, 0, (h)->stream>>>(__VA_ARGS__);                   \
    } else {                                                                             \
      if ((h)->q == 27) K<double, 27><<<grid, block, 0, (h)->stream>>>(__VA_ARGS__);     \
      else K<double, 19><<<grid, block, 0, (h)->stream>>>(__VA_ARGS__);                  \
    }                                                                                    \
  } while (0)

int check3(const lbm3d_config *cfg, std::string &err) {
  if (!cfg || cfg->n_members < 1 || !cfg->members) { err = "need n_members >= 1 and members"; return LBM_ERR_ARG; }
  if (cfg->precision != 32 && cfg->precision != 64) { err = "precision must be 32 or 64"; return LBM_ERR_ARG; }
  if (cfg->diag_every < 0) { err = "diag_every must be >= 0"; return LBM_ERR_ARG; }
  if (cfg->lattice != 0 && cfg->lattice != 19 && cfg->lattice != 27) { err = "lattice must be 19 or 27 (0: 19)"; return LBM_ERR_ARG; }
  if (cfg->diag_precision != 0 && cfg->diag_precision != 32 && cfg->diag_precision != 64) { err = "diag_precision must be 0, 32 or 64"; return LBM_ERR_ARG; }
  for (int m = 0; m < cfg->n_members; ++m) {
    const lbm3d_member_cfg &c = cfg->members[m];
    if (c.nx < 1 || c.ny < 1 || c.nz < 1 || (long long)c.nx * c.ny * c.nz > (1LL << 28)) { err = "grid out of range"; return LBM_ERR_ARG; }
    if (!(c.tau > 0.5) || !std::isfinite(c.tau)) { err = "tau must be > 0.5"; return LBM_ERR_ARG; }
    if (!(c.rho0 > 0.0) || !std::isfinite(c.rho0)) { err = "rho0 must be > 0"; return LBM_ERR_ARG; }
    if (c.force_kind != 0 && c.force_kind != 1) { err = "force_kind must be 0 or 1"; return LBM_ERR_ARG; }
    if (!std::isfinite(c.F0) || !std::isfinite(c.alpha)) { err = "F0/alpha not finite"; return LBM_ERR_ARG; }
  }
  return LBM_OK;
}

Layout3 layout3(const lbm3d_config *cfg) {
  Layout3 L{};
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off = al(off + b); return o; };
  const size_t es = cfg->precision == 32 ? 4 : 8;
  const size_t Q = lattice_q(cfg);
  L.members = take(sizeof(M3) * cfg->n_members);
  size_t Nmax = 0, Tmax = 0;
  for (int m = 0; m < cfg->n_members; ++m) {
    const lbm3d_member_cfg &c = cfg->members[m];
    const size_t N = (size_t)c.nx * c.ny * c.nz;
    L.pop0.push_back(take(es * Q * N));
    L.pop1.push_back(take(es * Q * N));
    L.snap.push_back(take(8 * 3 * 4 * N));
    L.ftab.push_back(take(es * (c.nx + c.ny + c.nz)));
    L.ftab64.push_back(take(8 * (c.nx + c.ny + c.nz)));
    Nmax = std::max(Nmax, N);
    Tmax = std::max(Tmax, (size_t)(c.nx + 1) * (c.ny + 1) * (c.nz + 1));
  }
  // fields, 13 tables (as int64), scales/means, query partials
  L.diag_doubles = (size_t)NF3 * Nmax + 13 * Tmax + 112 + (size_t)kMaxQBlocks3 * kQS3;
  L.diag = take(8 * L.diag_doubles);
  L.origin_cap = std::max<size_t>(3 * Nmax, (size_t)3 << 20);
  L.origins = take(4 * L.origin_cap);
  L.total = off;
  return L;
}

dim3 cells3(const lbm3d_member_cfg &c) { return dim3((c.nx + 63) / 64, (c.ny + 3) / 4, c.nz); }

int check_member3(lbm3d_handle *h, int m) {
  if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (m < 0 || m >= (int)h->mcfg.size()) return fail3(h, LBM_ERR_ARG, "member out of range");
  return LBM_OK;
}

bool snap_time3(const lbm3d_handle *h, long long t) {
  const long long D = h->cfg.diag_every;
  if (D <= 0) return false;
  const long long r = t % D;
  return r == 0 || r == D - 1 || r == D - 2;
}

int record3(lbm3d_handle *h) {
  const int slot = (int)(h->t % 3);
  for (int m = 0; m < (int)h->mcfg.size(); ++m)
    DISPATCH3(h, k3_snapshot, cells3(h->mcfg[m]), dim3(64, 4), h->d_m, m, h->cur, slot);
  CK3(cudaGetLastError());
  h->ring_time[slot] = h->t;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm3d_workspace_size(const lbm3d_config *cfg, size_t *bytes) {
  std::string err;
  if (int rc = check3(cfg, err)) return fail3(nullptr, rc, err);
  if (!bytes) return fail3(nullptr, LBM_ERR_ARG, "bytes is NULL");
  *bytes = layout3(cfg).total;
  return LBM_OK;
}

int lbm3d_create(const lbm3d_config *cfg, void *workspace, size_t bytes, lbm3d_handle **out) {
  std::string err;
  if (int rc = check3(cfg, err)) return fail3(nullptr, rc, err);
  if (!out) return fail3(nullptr, LBM_ERR_ARG, "out is NULL");
  const Layout3 L = layout3(cfg);
  if (!workspace || bytes < L.total || reinterpret_cast<uintptr_t>(workspace) % kAl)
    return fail3(nullptr, LBM_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  lbm3d_handle *h = new lbm3d_handle();
  h->cfg = *cfg;
  h->mcfg.assign(cfg->members, cfg->members + cfg->n_members);
  h->cfg.members = h->mcfg.data();
  h->ws = static_cast<char *>(workspace);
  h->ws_bytes = bytes;
  h->precision = cfg->precision;
  h->q = lattice_q(cfg);
  h->diag_prec = cfg->diag_precision == 32 ? 32 : 64;
  h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  h->d_m = reinterpret_cast<M3 *>(h->ws + L.members);
  h->diag = reinterpret_cast<double *>(h->ws + L.diag);
  h->diag_doubles = L.diag_doubles;
  h->d_origins = reinterpret_cast<int *>(h->ws + L.origins);
  h->origin_cap = L.origin_cap;
  const size_t es = cfg->precision == 32 ? 4 : 8;
  const size_t Q = h->q;
  for (int m = 0; m < cfg->n_members; ++m) {
    const lbm3d_member_cfg &c = h->mcfg[m];
    M3 M{};
    M.q = h->q;
    M.nx = c.nx;
    M.ny = c.ny;
    M.nz = c.nz;
    M.force_kind = c.force_kind;
    M.kf = c.kf;
    M.tau = c.tau;
    M.omega = 1.0 / c.tau;
    M.rho0 = c.rho0;
    M.F0 = c.F0;
    M.alpha = c.alpha;
    M.nu = (c.tau - 0.5) / 3.0;
    M.rho0_f = (float)c.rho0;
    M.omega_f = (float)(1.0 / c.tau);
    M.alpha_f = (float)c.alpha;
    M.F0_f = (float)c.F0;
    M.N = (size_t)c.nx * c.ny * c.nz;
    M.pop[0] = h->ws + L.pop0[m];
    M.pop[1] = h->ws + L.pop1[m];
    M.snap = reinterpret_cast<double *>(h->ws + L.snap[m]);
    M.ftab = h->ws + L.ftab[m];
    M.ftab64 = reinterpret_cast<double *>(h->ws + L.ftab64[m]);
    h->hm.push_back(M);
    // force tables: F_x(y), F_y(z), F_z(x)
    std::vector<double> ft(c.nx + c.ny + c.nz, 0.0);
    if (c.force_kind == 1) {
      const double pi = 3.14159265358979323846;
      for (int y = 0; y < c.ny; ++y) ft[y] = c.F0 * std::sin(2.0 * pi * c.kf * (double)y / c.ny);
      for (int z = 0; z < c.nz; ++z) ft[c.ny + z] = c.F0 * std::sin(2.0 * pi * c.kf * (double)z / c.nz);
      for (int x = 0; x < c.nx; ++x)
        ft[c.ny + c.nz + x] = c.F0 * std::sin(2.0 * pi * c.kf * (double)x / c.nx);
    }
    std::vector<float> ftf(ft.begin(), ft.end());
    cudaError_t e = cudaMemsetAsync(M.pop[0], 0, es * Q * M.N, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.pop[1], 0, es * Q * M.N, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(M.ftab64, ft.data(), 8 * ft.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = es == 8 ? cudaMemcpyAsync(M.ftab, ft.data(), 8 * ft.size(), cudaMemcpyHostToDevice, h->stream)
                  : cudaMemcpyAsync(M.ftab, ftf.data(), 4 * ftf.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // host tables are temporaries
    if (e != cudaSuccess) {
      delete h;
      return fail3(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  cudaError_t e = vec_layout(h, 4);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = tune_vec3(h);
  if (e != cudaSuccess) {
    delete h;
    return fail3(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = h;
  return LBM_OK;
}

int lbm3d_destroy(lbm3d_handle *h) {
  if (!h) return LBM_OK;  // like free(NULL)
  cudaStreamSynchronize(h->stream);
  delete h;
  return LBM_OK;
}

int lbm3d_init_fields(lbm3d_handle *h, int member, const double *rho, const double *ux,
                      const double *uy, const double *uz, int on_device) {
  if (int rc = check_member3(h, member)) return rc;
  if (!rho || !ux || !uy || !uz) return fail3(h, LBM_ERR_ARG, "fields must not be NULL");
  const M3 &M = h->hm[member];
  const double *src[4] = {rho, ux, uy, uz};
  double *dev[4];
  if (!on_device) {  // stage through the diagnostic scratch
    for (int q = 0; q < 4; ++q) {
      dev[q] = h->diag + (size_t)q * M.N;
      CK3(cudaMemcpyAsync(dev[q], src[q], 8 * M.N, cudaMemcpyHostToDevice, h->stream));
    }
  } else {
    for (int q = 0; q < 4; ++q) dev[q] = const_cast<double *>(src[q]);
  }
  DISPATCH3(h, k3_init, cells3(h->mcfg[member]), dim3(64, 4), h->d_m, member, h->cur, dev[0],
            dev[1], dev[2], dev[3]);
  CK3(cudaGetLastError());
  if (!on_device) CK3(cudaStreamSynchronize(h->stream));
  for (long long &r : h->ring_time) r = -1;
  return LBM_OK;
}

int lbm3d_step(lbm3d_handle *h, int nsteps) {
  if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (nsteps < 0) return fail3(h, LBM_ERR_ARG, "nsteps must be >= 0");
  for (int s = 0; s < nsteps; ++s) {
    if (snap_time3(h, h->t) && h->ring_time[h->t % 3] != h->t)
      if (int rc = record3(h)) return rc;
    if (h->vec_items > 0) launch_vec3(h, h->stream);  // every FP32 member with nx % 4 == 0
    for (int m = 0; m < (int)h->mcfg.size(); ++m)
      if (h->hm[m].items == 0)
        DISPATCH3(h, k3_step, cells3(h->mcfg[m]), dim3(64, 4), h->d_m, m, h->cur);
    CK3(cudaGetLastError());
    h->cur ^= 1;
    h->t += 1;
  }
  if (snap_time3(h, h->t) && h->ring_time[h->t % 3] != h->t) return record3(h);
  return LBM_OK;
}

long long lbm3d_time(const lbm3d_handle *h) { return h ? h->t : -1; }

int lbm3d_cells_per_lane(const lbm3d_handle *h) {
  return h ? (h->vec_items > 0 ? h->cpl : 0) : -1;
}

int lbm3d_set_cells_per_lane(lbm3d_handle *h, int cpl) {
  if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (cpl != 4 && cpl != 2) return fail3(h, LBM_ERR_ARG, "cells per lane must be 4 or 2");
  CK3(vec_layout(h, cpl));
  CK3(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm3d_get_populations(lbm3d_handle *h, int member, double *f, int on_device) {
  if (int rc = check_member3(h, member)) return rc;
  if (!f) return fail3(h, LBM_ERR_ARG, "f is NULL");
  const M3 &M = h->hm[member];
  double *dst = on_device ? f : h->diag;
  DISPATCH3(h, k3_copy, cells3(h->mcfg[member]), dim3(64, 4), h->d_m, member, h->cur, dst, 1);
  CK3(cudaGetLastError());
  if (!on_device) {
    CK3(cudaMemcpyAsync(f, dst, 8 * (size_t)h->q * M.N, cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

int lbm3d_set_populations(lbm3d_handle *h, int member, const double *f, int on_device) {
  if (int rc = check_member3(h, member)) return rc;
  if (!f) return fail3(h, LBM_ERR_ARG, "f is NULL");
  const M3 &M = h->hm[member];
  double *src = const_cast<double *>(f);
  if (!on_device) {
    src = h->diag;
    CK3(cudaMemcpyAsync(src, f, 8 * (size_t)h->q * M.N, cudaMemcpyHostToDevice, h->stream));
  }
  DISPATCH3(h, k3_copy, cells3(h->mcfg[member]), dim3(64, 4), h->d_m, member, h->cur, src, 0);
  CK3(cudaGetLastError());
  if (!on_device) CK3(cudaStreamSynchronize(h->stream));
  for (long long &r : h->ring_time) r = -1;
  return LBM_OK;
}

int lbm3d_record_snapshot(lbm3d_handle *h) {
  if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
  return record3(h);
}

int lbm3d_subvolume_balance(lbm3d_handle *h, int member, const int *L, int nL,
                            const int *origins, const int *counts, double *stats_out,
                            double *per_box_out) {
  if (int rc = check_member3(h, member)) return rc;
  if (!L || nL < 1 || nL > 32 || !stats_out) return fail3(h, LBM_ERR_ARG, "need 1..32 sizes and stats_out");
  if ((origins == nullptr) != (counts == nullptr))
    return fail3(h, LBM_ERR_ARG, "origins and counts go together");
  const lbm3d_member_cfg &c = h->mcfg[member];
  const M3 &M = h->hm[member];
  size_t total = 0;
  if (origins) {
    for (int i = 0; i < nL; ++i) {
      if (counts[i] < 1) return fail3(h, LBM_ERR_ARG, "every size needs a box");
      total += counts[i];
    }
    if (3 * total > h->origin_cap) return fail3(h, LBM_ERR_ARG, "too many boxes");
    for (size_t b = 0; b < total; ++b)
      if (origins[3 * b] < 0 || origins[3 * b] >= c.nx || origins[3 * b + 1] < 0 ||
          origins[3 * b + 1] >= c.ny || origins[3 * b + 2] < 0 || origins[3 * b + 2] >= c.nz)
        return fail3(h, LBM_ERR_ARG, "origin outside the grid");
  }
  const long long t = h->t;
  if (h->ring_time[t % 3] != t)
    if (int rc = record3(h)) return rc;
  if (t < 2 || h->ring_time[(t - 1) % 3] != t - 1 || h->ring_time[(t - 2) % 3] != t - 2)
    return fail3(h, LBM_ERR_HISTORY, "snapshots of time n-1 and n-2 are missing");
  const int Lmax = std::min(c.nx, std::min(c.ny, c.nz));
  if (per_box_out)
    for (int i = 0; i < nL; ++i)
      if (L[i] < 1 || L[i] > Lmax) return fail3(h, LBM_ERR_ARG, "per_box_out needs every size to fit");
  const size_t N = M.N;
  Diag3 J;
  J.m = h->d_m + member;
  J.s0 = M.snap + (size_t)(t % 3) * 4 * N;
  J.s1 = M.snap + (size_t)((t - 1) % 3) * 4 * N;
  J.s2 = M.snap + (size_t)((t - 2) % 3) * 4 * N;
  J.f = h->diag;
  const size_t T = (size_t)(c.nx + 1) * (c.ny + 1) * (c.nz + 1);
  long long *tab = reinterpret_cast<long long *>(h->diag + (size_t)NF3 * N);
  double *scales = h->diag + (size_t)NF3 * N + 13 * T;  // [16] scales, [16] exponents
  double *means = scales + 32;                           // [16]
  double *sd = scales + 48;                              // [30] statistics of one size
  // scales + 80: [16] inverse scales 2^-e; scales + 96: [16] maxima bit patterns
  double *partials = scales + 112;                       // [blocks][kQS3]
  const dim3 cb(64, 4), cg = cells3(c);
  unsigned long long *maxbits = reinterpret_cast<unsigned long long *>(scales + 96);
  CK3(cudaMemsetAsync(maxbits, 0, 16 * sizeof(unsigned long long), h->stream));
  const dim3 ag((unsigned)std::min<size_t>(256, (N + 2047) / 2048), 13);
  const dim3 sg((c.ny + 1 + 63) / 64, c.nz + 1, 13);
  if (h->diag_prec == 32) {  // term arithmetic in FP32
    k3_prep<float><<<cg, cb, 0, h->stream>>>(J);
    k3_grad<float><<<cg, cb, 0, h->stream>>>(J);
    k3_flux<float><<<cg, cb, 0, h->stream>>>(J);
    k3_curl<float><<<cg, cb, 0, h->stream>>>(J);
    k3_absmax<float><<<ag, 256, 0, h->stream>>>(J, maxbits);
    k3_scales<<<1, 32, 0, h->stream>>>(J, maxbits, scales);
    k3_scan_x<float><<<sg, 64, 0, h->stream>>>(J, scales, tab);
  } else {
    k3_prep<double><<<cg, cb, 0, h->stream>>>(J);
    k3_grad<double><<<cg, cb, 0, h->stream>>>(J);
    k3_flux<double><<<cg, cb, 0, h->stream>>>(J);
    k3_curl<double><<<cg, cb, 0, h->stream>>>(J);
    k3_absmax<double><<<ag, 256, 0, h->stream>>>(J, maxbits);
    k3_scales<<<1, 32, 0, h->stream>>>(J, maxbits, scales);
    k3_scan_x<double><<<sg, 64, 0, h->stream>>>(J, scales, tab);
  }
  k3_scan_yz<<<dim3((c.nx + 1 + 63) / 64, c.nz + 1, 13), 64, 0, h->stream>>>(J, tab, 1);
  k3_scan_yz<<<dim3((c.nx + 1 + 63) / 64, c.ny + 1, 13), 64, 0, h->stream>>>(J, tab, 2);
  k3_means<<<1, 32, 0, h->stream>>>(J, tab, scales, means);
  CK3(cudaGetLastError());
  if (origins)
    CK3(cudaMemcpyAsync(h->d_origins, origins, 12 * total, cudaMemcpyHostToDevice, h->stream));
  std::vector<double> host(30 * (size_t)nL, std::nan(""));
  size_t ooff = 0, row = 0;
  for (int i = 0; i < nL; ++i) {
    const int nb = origins ? counts[i] : (int)N;
    if (L[i] >= 1 && L[i] <= Lmax) {
      const int qb = std::min(kMaxQBlocks3, std::max(1, (nb + 255) / 256));
      const int *og = origins ? h->d_origins + 3 * ooff : nullptr;
      double *pbo = per_box_out ? per_box_out + row * 15 : nullptr;
      if (h->diag_prec == 32)
        k3_query<float><<<qb, 256, 0, h->stream>>>(J, tab, scales, means, L[i], nb, og, partials,
                                                   pbo);
      else
        k3_query<double><<<qb, 256, 0, h->stream>>>(J, tab, scales, means, L[i], nb, og,
                                                    partials, pbo);
      k3_stats<<<1, 15 * 32, 0, h->stream>>>(partials, qb, means, nb, sd);
      CK3(cudaGetLastError());
      CK3(cudaMemcpyAsync(host.data() + 30 * (size_t)i, sd, 8 * 30, cudaMemcpyDeviceToHost,
                          h->stream));
    }
    ooff += origins ? counts[i] : 0;
    row += nb;
  }
  CK3(cudaStreamSynchronize(h->stream));
  std::copy(host.begin(), host.end(), stats_out);
  return LBM_OK;
}

const char *lbm3d_last_error(const lbm3d_handle *h) {
  return h ? h->err.c_str() : g_err3.c_str();
}

}  // extern "C"
