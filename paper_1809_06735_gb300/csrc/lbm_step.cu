// D2Q9 BGK stream-collide with exact-difference forcing (eq. (1), eq. (2),
// Sec. 3 of Tauzin et al. 2018) and the kernels that move the state in and
// out of the device storage (see lbm_internal.cuh).
//
// Storage states (an int carried by the handle and flipped by each step):
//   0, 1  double buffer, pull layout: buffer `state` holds post-collision
//         values at their origin cell; f_l(x, n) = pop[state][l][x - c_l];
//         a step reads buffer `state` and writes the other one.
//   2     in-place AA layout, even phase: f_l(x, n) = pop[0][l][x];
//         the step reads slot l at x and writes f*_l(x) to slot opposite(l)
//         at x (no neighbour access at all).
//   3     in-place AA layout, odd phase: f_l(x, n) = pop[0][opposite(l)][x - c_l];
//         the step reads there and writes f*_l(x) to slot l at x + c_l, which
//         is the even-phase location of f_l(x + c_l, n + 1).
// In the odd phase each location is read and then written by the same cell
// (slot opposite(l) at x - c_l is slot m = opposite(l) at x + c_m), so the
// in-place update has no race.  Both layouts move 72 B per FP32 lattice
// update; AA needs one population array instead of two.
//
// Hot kernel: k_step_f32_vec, one launch per time step over every member of
// the ensemble.  Each warp owns 128 consecutive cells of one row (4 per
// lane); each of the 9 populations is one aligned 128-bit load per lane from
// its source row, and the +-1 shift of the x-moving populations is a warp
// shuffle with one scalar load at each warp edge (the AA odd phase does the
// same for its shifted stores), so DRAM sees coalesced 16-byte accesses.
#include "lbm_internal.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Collision of one cell.
// ---------------------------------------------------------------------------

// FP32 deviation form: g_l = f_l - t_l rho0.  rho = rho0 + sum g,
// j = sum c g.  g_eq_l = t_l [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)];
// EDM term F_l = f_eq_l(rho, u + du) - f_eq_l(rho, u) written as
// t_l rho [3 c.du + 4.5 c.du (2 c.u + c.du) - 1.5 du.(2u + du)], du = F/rho,
// F = F_ext - alpha j.  Post-collision g_l - omega (g_l - g_eq_l) + F_l.
// Local relaxation time of the variable-viscosity collisions in deviation
// form: Pi^neq = sum c c g - drho cs^2 I - rho u u (moments as collide_f32
// forms them, so the snapshot's viscosity is the one the step used).
__device__ __forceinline__ float local_tau_f32(const float g[kQ], float drho, float rho, float ux,
                                               float uy, float tau0, int coll, float Cs) {
  const float d4 = (g[5] + g[6]) + (g[7] + g[8]);
  const float pxx = (g[1] + g[3]) + d4 - drho * (1.0f / 3.0f) - rho * ux * ux;
  const float pyy = (g[2] + g[4]) + d4 - drho * (1.0f / 3.0f) - rho * uy * uy;
  const float pxy = (g[5] - g[6]) + (g[7] - g[8]) - rho * ux * uy;
  return tau_from_stress<float>(pxx, pxy, pyy, rho, tau0, coll, Cs);
}
__device__ __forceinline__ void moments_f32(const float g[kQ], float rho0, float &drho,
                                            float &rho, float &jx, float &jy, float &ir,
                                            float &ux, float &uy) {
  drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
  jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
  rho = rho0 + drho;
  ir = 1.0f / rho;
  ux = jx * ir;
  uy = jy * ir;
}
// FP64: Pi^neq = sum c c f - rho cs^2 I - rho u u.
__device__ __forceinline__ double local_tau_f64(const double f[kQ], double rho, double ux,
                                                double uy, double tau0, int coll, double Cs) {
  double sxx = 0.0, sxy = 0.0, syy = 0.0;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    if (cx_of(l) != 0) sxx += f[l];
    if (cx_of(l) * cy_of(l) != 0) sxy += cx_of(l) * cy_of(l) * f[l];
    if (cy_of(l) != 0) syy += f[l];
  }
  return tau_from_stress<double>(sxx - rho / 3.0 - rho * ux * ux, sxy - rho * ux * uy,
                                 syy - rho / 3.0 - rho * uy * uy, rho, tau0, coll, Cs);
}
__device__ __forceinline__ void moments_f64(const double f[kQ], double &rho, double &ux,
                                            double &uy) {
  double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {  // terms with c = 0 skipped (a product by 0 is not
    r += f[l];                       // dropped by IEEE arithmetic: it costs an FMA)
    if (cx_of(l) != 0) jx += cx_of(l) * f[l];
    if (cy_of(l) != 0) jy += cy_of(l) * f[l];
  }
  rho = r;
  const double ir = 1.0 / r;
  ux = jx * ir;
  uy = jy * ir;
}

// ---------------------------------------------------------------------------
// Entropic LBM (collision 3): the equilibrium minimising H = sum f ln(f/t),
// the non-trivial root alpha of H(f + alpha Delta) = H(f), Delta = f_eq - f,
// f' = f + alpha Delta / (2 tau0) + F_l (EDM on the same equilibrium).
// ---------------------------------------------------------------------------

// phi(z) = (1 + z) ln(1 + z) - z: series where the terms cancel.
// ln(1 + z) for the FP32 entropic collision, whose arguments are mostly
// small (relative populations' departures): its Taylor series in Horner
// form where |z| < 1/8 (the terms after z^9 / 9 are below 1e-10 of |z|,
// under the FP32 rounding), the library function elsewhere.  FP64 keeps the
// library functions.
__device__ __forceinline__ float ln1p_series(float z) {
  float p = 1.0f / 9.0f;
  p = fmaf(-z, p, 1.0f / 8.0f);
  p = fmaf(-z, p, 1.0f / 7.0f);
  p = fmaf(-z, p, 1.0f / 6.0f);
  p = fmaf(-z, p, 1.0f / 5.0f);
  p = fmaf(-z, p, 1.0f / 4.0f);
  p = fmaf(-z, p, 1.0f / 3.0f);
  p = fmaf(-z, p, 1.0f / 2.0f);
  p = fmaf(-z, p, 1.0f);
  return z * p;
}
template <typename T>
__device__ __forceinline__ T ln1p_e(T z) {
  if constexpr (sizeof(T) == 4)
    return fabsf(z) < 0.125f ? ln1p_series(z) : log1pf(z);
  else
    return log1p(z);
}

// a / b for the entropic collision: FP32 with the fast division intrinsic
// (at most 2 ulp; every denominator here is a population, a density or a
// sum of order one), FP64 exact.
template <typename T>
__device__ __forceinline__ T div_e(T a, T b) {
  if constexpr (sizeof(T) == 4)
    return __fdividef(a, b);
  else
    return a / b;
}

template <typename T>
__device__ __forceinline__ T phi_entropy(T z) {
  const T lim = sizeof(T) == 4 ? T(0.1) : T(0.1);
  if (fabs(z) < lim) {
    const int K = sizeof(T) == 4 ? 10 : 24;
    T s = T(0), p = z * z;
#pragma unroll
    for (int k = 2; k < K; ++k) {
      s += ((k & 1) ? -p : p) * T(1.0 / (k * (k - 1)));
      p *= z;
    }
    return s;
  }
  return (T(1) + z) * ln1p_e<T>(z) - z;
}

// g(a) = sum f phi(a y) - a S2, y = Delta / f, S2 = sum Delta ln(1 + y);
// *scale (if given) receives the magnitude of the terms, the size of g's
// rounding noise.
template <typename T>
__device__ __forceinline__ T entropy_gap(const T f[kQ], const T y[kQ], T S2, T a,
                                         T *scale = nullptr) {
  T s = T(0);
#pragma unroll
  for (int l = 0; l < kQ; ++l) s += f[l] * phi_entropy<T>(a * y[l]);
  if (scale) *scale = s + a * fabs(S2);
  return s - a * S2;
}

// The root alpha > 1 (alpha = 2 at equilibrium, for non-positive populations
// or without a root below min(a_max, 64)).  FP64: bisection to 1e-15 (the
// oracle's procedure); FP32: the third-order series of the root in the
// populations' relative departures y when every |y| < 0.02 (error below
// 1e-7), otherwise Newton from that series, g'(a) = sum Delta ln(1 + a y) -
// S2, kept inside a bisection bracket, until |g| is at the level of its
// rounding (1e-6 of the terms; then one last Newton step if it stays in the
// bracket) or a step below 1e-3 a (error of order 1e-6 a after it).
template <typename T>
__device__ T elbm_alpha(const T f[kQ], const T d[kQ]) {
  T y[kQ], ymax = T(0), S2 = T(0);
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    if (!(f[l] > T(0))) return T(2);
    y[l] = div_e<T>(d[l], f[l]);
    ymax = fmax(ymax, fabs(y[l]));
  }
  if (ymax < (sizeof(T) == 4 ? T(1e-7) : T(1e-12))) return T(2);
  // the bracket (1, a_max): f + a Delta stays positive below a_max
  auto upper = [&]() {
    T amax = T(64);
#pragma unroll
    for (int l = 0; l < kQ; ++l)
      if (y[l] < T(0)) amax = fmin(amax, div_e<T>(-T(1), y[l]));
    return amax * (sizeof(T) == 4 ? T(1 - 1e-6) : T(1 - 1e-12));
  };
  T lo = T(1), hi;
  if constexpr (sizeof(T) == 8) {
    hi = upper();
#pragma unroll
    for (int l = 0; l < kQ; ++l) S2 += d[l] * ln1p_e<T>(y[l]);
    if (entropy_gap<T>(f, y, S2, hi) < T(0)) return T(2);
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
      const T mid = T(0.5) * (lo + hi);
      if (entropy_gap<T>(f, y, S2, mid) < T(0))
        lo = mid;
      else
        hi = mid;
    }
    return T(0.5) * (lo + hi);
  } else {
    // The root as a series in y = Delta / f about the BGK value a = 2: with
    // T_k = sum_l f_l y_l^k (of order y^k), the entropy condition g(a) / a
    // = sum_{k>=2} (-1)^k T_k (a^(k-1) - k) / (k (k - 1)) = 0 solved order
    // by order in y gives a = 2 + c1 + c2 + c3 + O(y^4),
    //   c1 = u / 3, c2 = 4 u^2 / 9 - 2 q4 / 3,
    //   c3 = 11 q5 / 10 - 14 u q4 / 9 + 17 u^3 / 27,
    // u = T3 / T2, q4 = T4 / T2, q5 = T5 / T2.  Against the root of the
    // entropy condition to 40 digits its error is below 1e-7 (under the FP32
    // rounding of a) while max |y| < 0.02: the series is then the root.
    // Otherwise it starts Newton's iteration on g.
    T T2 = T(0), T3 = T(0), T4 = T(0), T5 = T(0);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {  // f y^k = Delta y^(k-1)
      const T y2 = y[l] * y[l], dy2 = d[l] * y2;
      T2 = fma(d[l], y[l], T2);
      T3 = fma(d[l], y2, T3);
      T4 = fma(dy2, y[l], T4);
      T5 = fma(dy2, y2, T5);
    }
    const T r2 = div_e<T>(T(1), T2), u = T3 * r2, q4 = T4 * r2, q5 = T5 * r2;
    T a = T(2) + (u * T(1.0 / 3.0) + (T(4.0 / 9.0) * u * u - T(2.0 / 3.0) * q4 +
                                      T(1.1) * q5 - T(14.0 / 9.0) * u * q4 +
                                      T(17.0 / 27.0) * u * u * u));
    if (ymax < T(0.02)) return a;
    hi = upper();
#pragma unroll
    for (int l = 0; l < kQ; ++l) S2 += d[l] * ln1p_e<T>(y[l]);
    if (!(a > lo && a < hi)) a = fmin(T(2), T(0.5) * (lo + hi));
    bool bracketed = false;
    for (int it = 0; it < 30; ++it) {
      // g(a) and g'(a) = sum Delta ln(1 + a y) - S2 share ln(1 + a y): one
      // log1p per population (phi as entropy_gap evaluates it)
      T s = T(0), dg = -S2;
#pragma unroll
      for (int l = 0; l < kQ; ++l) {
        const T z = a * y[l], lz = ln1p_e<T>(z);
        T ph;
        if (fabs(z) < T(0.1)) {
          // phi(z) = sum_{k>=2} (-1)^k z^k / (k (k - 1)), terms to z^9, in
          // Horner form
          T p = T(1.0 / 72.0);
#pragma unroll
          for (int k = 8; k >= 2; --k) p = fma(-z, p, T(1.0 / (k * (k - 1))));
          ph = z * z * p;
        } else {
          ph = (T(1) + z) * lz - z;
        }
        s += f[l] * ph;
        dg += d[l] * lz;
      }
      const T scale = s + a * fabs(S2);
      const T g = s - a * S2;
      const bool conv = fabs(g) <= T(1e-6) * scale;
      if (g < T(0))
        lo = a;
      else
        hi = a;
      T an = a - div_e<T>(g, dg);
      const bool inside = an > lo && an < hi;
      if (conv) return inside ? an : a;
      // Newton on the convex g converges quadratically: a step below 1e-3 a
      // leaves an error of order 1e-6 a, the FP32 rounding level of the root
      if (inside && fabs(an - a) < T(1e-3) * a) return an;
      if (!bracketed) {  // no root below the positivity limit: the BGK value
        bracketed = true;
        if (entropy_gap<T>(f, y, S2, hi) < T(0)) return T(2);
      }
      if (!inside) an = T(0.5) * (lo + hi);  // left the bracket: bisect
      const bool done = fabs(an - a) < T(1e-6) * a;
      a = an;
      if (done) break;
    }
    return a;
  }
}

// ln of the entropic equilibrium's velocity factor, per population (FP64):
// ln P_l(u) = sum_a [ln(2 - s_a) + c_la ln((2 u_a + s_a) / (1 - u_a))],
// s_a = sqrt(1 + 3 u_a^2), each logarithm as log1p of a cancellation-free
// argument (s - 1 = 3 u^2 / (1 + s)).
template <typename T>
__device__ __forceinline__ void entropic_logp(T ux, T uy, T lp[kQ]) {
  const T sx = sqrt(T(1) + T(3) * ux * ux), sy = sqrt(T(1) + T(3) * uy * uy);
  const T qx = div_e<T>(T(3) * ux * ux, T(1) + sx), qy = div_e<T>(T(3) * uy * uy, T(1) + sy);
  const T a0x = ln1p_e<T>(-qx), a0y = ln1p_e<T>(-qy);
  const T a1x = ln1p_e<T>(div_e<T>(T(3) * ux + qx, T(1) - ux));
  const T a1y = ln1p_e<T>(div_e<T>(T(3) * uy + qy, T(1) - uy));
#pragma unroll
  for (int l = 0; l < kQ; ++l)
    lp[l] = a0x + a0y + (T)cx_of(l) * a1x + (T)cy_of(l) * a1y;
}

// P_l(u) - 1 for FP32 from the product form of the same factor,
// P_l = prod_a (2 - s_a) ((2 u_a + s_a) / (1 - u_a))^(c_la): with
// q = s - 1 = 3 u^2 / (1 + s), the factor of an axis is 1 + Z_c for
// c = 0, +1, -1: Z_0 = -q, Z_(+1) = b - q - q b with b = (3 u + q) / (1 - u),
// Z_(-1) = b' - q - q b' with b' = -(3 u + q) / (1 + 2 u + q), and
// P - 1 = X + Y + X Y: no logarithm or exponential, no cancellation.
__device__ __forceinline__ void entropic_em_f32(float ux, float uy, float em[kQ]) {
  float X[3], Y[3];  // indexed by c + 1
  auto axis = [](float u, float (&Z)[3]) {
    const float s = sqrtf(1.0f + 3.0f * u * u);
    const float q = __fdividef(3.0f * u * u, 1.0f + s);
    const float n = 3.0f * u + q;
    const float b = __fdividef(n, 1.0f - u), bm = -__fdividef(n, 1.0f + 2.0f * u + q);
    Z[0] = fmaf(-q, bm, bm - q);
    Z[1] = -q;
    Z[2] = fmaf(-q, b, b - q);
  };
  axis(ux, X);
  axis(uy, Y);
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const float x = X[cx_of(l) + 1], y = Y[cy_of(l) + 1];
    em[l] = fmaf(x, y, x + y);
  }
}

// One ELBM collision in storage form (FP32: deviations g = f - t rho0, FP64:
// f); returns alpha.
template <typename T>
__device__ T collide_elbm(T v[kQ], T rho0, T tau0, T Fex, T Fey, T alpha_drag) {
  T rho, jx, jy, drho, ux, uy;
  if constexpr (sizeof(T) == 4) {
    float ir;
    moments_f32(v, rho0, drho, rho, jx, jy, ir, ux, uy);
  } else {
    rho = T(0);
    jx = T(0);
    jy = T(0);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      rho += v[l];
      if (cx_of(l) != 0) jx += cx_of(l) * v[l];
      if (cy_of(l) != 0) jy += cy_of(l) * v[l];
    }
    drho = T(0);
    ux = jx / rho;
    uy = jy / rho;
  }
  const T Fx = Fex - alpha_drag * jx, Fy = Fey - alpha_drag * jy;
  // without force the shifted velocity is u itself and the EDM term is
  // exactly zero: its second equilibrium is skipped
  const bool forced = Fx != T(0) || Fy != T(0);
  T f[kQ], d[kQ], Fl[kQ];
  if constexpr (sizeof(T) == 4) {
    float em[kQ], ems[kQ];  // P_l - 1 at u and at the shifted velocity
    entropic_em_f32(ux, uy, em);
    if (forced) entropic_em_f32(ux + div_e<T>(Fx, rho), uy + div_e<T>(Fy, rho), ems);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const float t = w_of(l);
      f[l] = fmaf(t, rho0, v[l]);
      // f_eq - f = t rho (1 + em) - t rho0 - v = t (drho + rho em) - v
      d[l] = fmaf(t, fmaf(rho, em[l], drho), -v[l]);
      Fl[l] = forced ? t * rho * (ems[l] - em[l]) : 0.0f;
    }
  } else {
    T lp[kQ], lps[kQ];
    entropic_logp<T>(ux, uy, lp);
    if (forced) entropic_logp<T>(ux + div_e<T>(Fx, rho), uy + div_e<T>(Fy, rho), lps);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const T t = (T)w_of(l);
      const T em = expm1(lp[l]);  // P_l - 1
      f[l] = v[l];
      d[l] = t * rho * (T(1) + em) - v[l];
      Fl[l] = forced ? t * rho * (T(1) + em) * expm1(lps[l] - lp[l]) : T(0);
    }
  }
  const T a = elbm_alpha<T>(f, d);
  const T ab = div_e<T>(a, T(2) * tau0);
  if (forced) {
#pragma unroll
    for (int l = 0; l < kQ; ++l) v[l] = v[l] + ab * d[l] + Fl[l];
  } else {
#pragma unroll
    for (int l = 0; l < kQ; ++l) v[l] = v[l] + ab * d[l];
  }
  return a;
}

// Relaxation time 2 tau0 / alpha of the ELBM state v (storage form).
template <typename T>
__device__ T elbm_tau(const T v[kQ], T rho0, T tau0) {
  T w[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) w[l] = v[l];
  const T a = collide_elbm<T>(w, rho0, tau0, T(0), T(0), T(0));
  return T(2) * tau0 / a;
}

// With VV (variable viscosity, collision != 0) omega = 1 / local_tau_f32.
template <bool VV = false>
__device__ __forceinline__ void collide_f32(float g[kQ], float rho0, float om, float Fex,
                                            float Fey, float alpha, int coll = 0,
                                            float tau0 = 0.f, float Cs = 0.f) {
  float drho, rho, jx, jy, ir, ux, uy;
  moments_f32(g, rho0, drho, rho, jx, jy, ir, ux, uy);
  if constexpr (VV) {
    if (coll != 0) om = 1.0f / local_tau_f32(g, drho, rho, ux, uy, tau0, coll, Cs);
  }
  const float Fx = Fex - alpha * jx, Fy = Fey - alpha * jy;
  const float dux = Fx * ir, duy = Fy * ir;
  const float usq = ux * ux + uy * uy;
  const float dsq = dux * (2.0f * ux + dux) + duy * (2.0f * uy + duy);
  const float base_eq = drho - 1.5f * rho * usq;  // t-scaled later
  const float base_F = -1.5f * rho * dsq;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const float t = (float)w_of(l);
    const float cu = (float)cx_of(l) * ux + (float)cy_of(l) * uy;
    const float cd = (float)cx_of(l) * dux + (float)cy_of(l) * duy;
    const float geq = t * (base_eq + rho * cu * (3.0f + 4.5f * cu));
    const float Fl = t * (base_F + rho * cd * (3.0f + 4.5f * (2.0f * cu + cd)));
    g[l] = g[l] - om * (g[l] - geq) + Fl;
  }
}

// FP64 plain form on the full populations f_l; coll != 0: omega from the
// local relaxation time (Pi^neq = sum c c f - rho cs^2 I - rho u u).
// The populations go in opposite pairs (l, opp(l)), c_opp = -c_l: the
// equilibrium and the exact-difference term split into a part even in c
// (the same for both) and an odd part (opposite signs), each formed once:
//   feq = t rho [1 - 1.5 |u|^2 + 4.5 (c.u)^2] +- 3 t rho |c.u|,
//   F_l = t rho [9 (c.u)(c.du) + 4.5 (c.du)^2 - 1.5 (2 u.du + |du|^2)] +- 3 t rho |c.du|,
// (du = F / rho), which halves the FP64 work (FP64 is this part's slow pipe).
// The relaxed sums om feq + F are formed before the common factor t rho:
//   e = t rho [om (base + 4.5 (c.u)^2) + (c.du) (4.5 c.du + 9 c.u) + mdsq],
//   o = 3 t rho (om c.u + c.du),  mdsq = -1.5 (2 u.du + |du|^2),
// 13 FP64 operations per pair.
__device__ __forceinline__ void collide_pair_f64(double &fp, double &fm, double cu, double cd,
                                                 double trho, double trho3, double base,
                                                 double mdsq, double om, double keep) {
  const double e = trho * fma(om, fma(4.5 * cu, cu, base), fma(cd, fma(4.5, cd, 9.0 * cu), mdsq));
  const double o = trho3 * fma(om, cu, cd);
  fp = fma(keep, fp, e + o);
  fm = fma(keep, fm, e - o);
}

__device__ __forceinline__ void collide_f64(double f[kQ], double om, double Fex, double Fey,
                                            double alpha, int coll = 0, double tau0 = 0.0,
                                            double Cs = 0.0) {
  const double rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const double jx = (f[1] + f[5] + f[8]) - (f[3] + f[6] + f[7]);
  const double jy = (f[2] + f[5] + f[6]) - (f[4] + f[7] + f[8]);
  const double ir = 1.0 / rho;
  const double ux = jx * ir, uy = jy * ir;
  if (coll != 0) om = 1.0 / local_tau_f64(f, rho, ux, uy, tau0, coll, Cs);
  const double Fx = Fex - alpha * jx, Fy = Fey - alpha * jy;
  const double dux = Fx * ir, duy = Fy * ir;
  const double usq = ux * ux + uy * uy;
  const double dsq = dux * (2.0 * ux + dux) + duy * (2.0 * uy + duy);
  const double base = 1.0 - 1.5 * usq, keep = 1.0 - om, mdsq = -1.5 * dsq;
  const double r0 = (4.0 / 9.0) * rho, r1 = (1.0 / 9.0) * rho, r2 = (1.0 / 36.0) * rho;
  const double r13 = (1.0 / 3.0) * rho, r23 = (1.0 / 12.0) * rho;  // 3 t rho
  // rest population: no odd part
  f[0] = fma(keep, f[0], r0 * fma(om, base, mdsq));
  collide_pair_f64(f[1], f[3], ux, dux, r1, r13, base, mdsq, om, keep);
  collide_pair_f64(f[2], f[4], uy, duy, r1, r13, base, mdsq, om, keep);
  collide_pair_f64(f[5], f[7], ux + uy, dux + duy, r2, r23, base, mdsq, om, keep);
  collide_pair_f64(f[6], f[8], uy - ux, duy - dux, r2, r23, base, mdsq, om, keep);
}

// Compensated FP32 sum of FP32 values as the unevaluated pair (s, c): the
// FP64 sum is (double)s + (double)c (the csum value) and differences of
// nearby sums can be formed in FP32 as (s - s') + (c - c').
__device__ __forceinline__ void csum_pair(const float *v, const int *sign, int n, float &s,
                                          float &c) {
  s = sign[0] * v[0];
  c = 0.f;
  for (int k = 1; k < n; ++k) {
    float e;
    two_sum(s, sign[k] * v[k], s, e);
    c += e;
  }
}

// ---------------------------------------------------------------------------
// Hot kernel: batched FP32 stream-collide, 4 cells per lane, nx % 4 == 0.
// blockDim = (32, WY); a tile is 128 x (WY * ROWS) cells of one member.
// MODE 0: double-buffer pull; 1: AA even phase; 2: AA odd phase.
// ---------------------------------------------------------------------------

// External force of 4 consecutive cells (x .. x+3, x % 4 == 0) of row y for
// force kind 2: the shell force table plus the damping of eq. (16) from the
// member's coefficients of this step.
__device__ __forceinline__ void paper_force4(const Member &M, int x, int y, float (&fx)[4],
                                             float (&fy)[4]) {
  const float *ft = static_cast<const float *>(M.ft_tab) + (size_t)y * M.pitch + x;
  const float4 tx = __ldg(reinterpret_cast<const float4 *>(ft));
  const float4 ty = __ldg(reinterpret_cast<const float4 *>(ft + M.plane));
  const float *tr = static_cast<const float *>(M.trig);
  const int nx = M.nx;
  const float4 cx = __ldg(reinterpret_cast<const float4 *>(tr + x));
  const float4 sx = __ldg(reinterpret_cast<const float4 *>(tr + nx + x));
  const float4 c2x = __ldg(reinterpret_cast<const float4 *>(tr + 2 * nx + x));
  const float4 s2x = __ldg(reinterpret_cast<const float4 *>(tr + 3 * nx + x));
  const float *row = M.damp_rows + 6 * (size_t)y;  // (P, Q, R) of x, then of y
  const float bx[4] = {tx.x, tx.y, tx.z, tx.w}, by[4] = {ty.x, ty.y, ty.z, ty.w};
  const float cxa[4] = {cx.x, cx.y, cx.z, cx.w}, sxa[4] = {sx.x, sx.y, sx.z, sx.w};
  const float c2xa[4] = {c2x.x, c2x.y, c2x.z, c2x.w}, s2xa[4] = {s2x.x, s2x.y, s2x.z, s2x.w};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float P = row[3 * k], Q = row[3 * k + 1], R = row[3 * k + 2];
    const float A4 = M.damp_f[12 * k + 8], B4 = M.damp_f[12 * k + 9];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float v = (k ? by[i] : bx[i]) + P * cxa[i] + Q * sxa[i] + A4 * c2xa[i] +
                      B4 * s2xa[i] + R;
      if (k)
        fy[i] = v;
      else
        fx[i] = v;
    }
  }
}

// One tile of the stream-collide: 128 x (blockDim.y * ROWS) cells of one
// member, 4 consecutive cells per lane.  SNAP: the step also records the
// snapshot-ring entry of the state it reads (slot snap_slot), the same
// compensated pairs as k_snapshot_ring.
template <int ROWS, int MODE, int PF, bool SNAP>
__device__ __forceinline__ void step_tile(const Member *__restrict__ members, const Tile tl,
                                          int cur, int snap_slot) {
  const int lane = threadIdx.x;
  const Member &M = members[tl.member];
  const int nx = M.nx, ny = M.ny, pitch = M.pitch;
  const size_t plane = M.plane;
  const float *src = static_cast<const float *>(MODE == 0 ? M.pop[cur] : M.pop[0]);
  float *dst = static_cast<float *>(MODE == 0 ? M.pop[cur ^ 1] : M.pop[0]);
  const float *__restrict__ fxt = static_cast<const float *>(M.fx_tab);
  const float *__restrict__ fyt = static_cast<const float *>(M.fy_tab);
  const float rho0 = M.rho0_f, om = M.omega_f, alpha = M.alpha_f;
  const int x = tl.x0 + 4 * lane;
  const bool active = x < nx;
  const bool last = active && (lane == 31 || x + 4 >= nx);  // last active lane of the row segment
  float4 fy4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (active) fy4 = *reinterpret_cast<const float4 *>(fyt + x);
  const float fy[4] = {fy4.x, fy4.y, fy4.z, fy4.w};
  const int xprev = (x == 0) ? nx - 1 : x - 1;  // cell left of the chunk
  const int xnext = (x + 4 >= nx) ? 0 : x + 4;  // cell right of the chunk

#pragma unroll 1
  for (int r = 0; r < ROWS; ++r) {
    const int y = tl.y0 + threadIdx.y * ROWS + r;
    if (y >= ny) break;  // uniform per warp
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y + 1 == ny) ? 0 : y + 1;
    float v[kQ][4];
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const int cxl = cx_of(l), cyl = cy_of(l);
      if (MODE == 1) {  // own cell, own slot
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active)
          o = __ldg(reinterpret_cast<const float4 *>(src + (size_t)l * plane +
                                                     (size_t)y * pitch + x));
        v[l][0] = o.x; v[l][1] = o.y; v[l][2] = o.z; v[l][3] = o.w;
        continue;
      }
      const int slot = MODE == 2 ? opposite(l) : l;
      const int ys = cyl == 0 ? y : (cyl > 0 ? ym : yp);  // pull from y - c_y
      const float *row = src + (size_t)slot * plane + (size_t)ys * pitch;
      // read-only (non-coherent) loads only when source and destination
      // differ; the in-place phase reads what it later overwrites
      float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
      if (active)
        o = MODE == 0 ? __ldg(reinterpret_cast<const float4 *>(row + x))
                      : *reinterpret_cast<const float4 *>(row + x);
      if (cxl == 0) {
        v[l][0] = o.x; v[l][1] = o.y; v[l][2] = o.z; v[l][3] = o.w;
      } else if (cxl > 0) {  // pull from x - 1
        float prev = __shfl_up_sync(0xffffffffu, o.w, 1);
        if (active && (lane == 0 || x == 0)) prev = MODE == 0 ? __ldg(row + xprev) : row[xprev];
        v[l][0] = prev; v[l][1] = o.x; v[l][2] = o.y; v[l][3] = o.z;
      } else {  // pull from x + 1
        float next = __shfl_down_sync(0xffffffffu, o.x, 1);
        if (last) next = MODE == 0 ? __ldg(row + xnext) : row[xnext];
        v[l][0] = o.y; v[l][1] = o.z; v[l][2] = o.w; v[l][3] = next;
      }
    }
    if constexpr (SNAP) {
      if (active) {  // (rho - rho0, j_x, j_y) of f(., n) as compensated pairs
        float hs[3][4], ls[3][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int one[kQ] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
          const int sgn[6] = {1, 1, 1, -1, -1, -1};
          float f[kQ];
#pragma unroll
          for (int l = 0; l < kQ; ++l) f[l] = v[l][c];
          const float ax[6] = {f[1], f[5], f[8], f[3], f[6], f[7]};
          const float ay[6] = {f[2], f[5], f[6], f[4], f[7], f[8]};
          csum_pair(f, one, kQ, hs[0][c], ls[0][c]);
          csum_pair(ax, sgn, 6, hs[1][c], ls[1][c]);
          csum_pair(ay, sgn, 6, hs[2][c], ls[2][c]);
        }
        const size_t N = (size_t)nx * ny;
        float *d = reinterpret_cast<float *>(M.snap) + (size_t)snap_slot * 6 * N +
                   (size_t)y * nx + x;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          __stcs(reinterpret_cast<float4 *>(d + (size_t)(2 * q) * N),
                 make_float4(hs[q][0], hs[q][1], hs[q][2], hs[q][3]));
          __stcs(reinterpret_cast<float4 *>(d + (size_t)(2 * q + 1) * N),
                 make_float4(ls[q][0], ls[q][1], ls[q][2], ls[q][3]));
        }
      }
    }
    if (active) {
      float fxc[4], fyc[4];
      if (PF != 0 && M.force_kind == 2) {
        paper_force4(M, x, y, fxc, fyc);
      } else {
        const float fx = fxt[y];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          fxc[c] = fx;
          fyc[c] = fy[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float g[kQ];
#pragma unroll
        for (int l = 0; l < kQ; ++l) g[l] = v[l][c];
        if constexpr (PF == 3) {
          if (M.collision == 3)
            collide_elbm<float>(g, rho0, M.tau_f, fxc[c], fyc[c], alpha);
          else
            collide_f32<true>(g, rho0, om, fxc[c], fyc[c], alpha, M.collision, M.tau_f, M.Cs_f);
        } else if constexpr (PF == 2)
          collide_f32<true>(g, rho0, om, fxc[c], fyc[c], alpha, M.collision, M.tau_f, M.Cs_f);
        else
          collide_f32(g, rho0, om, fxc[c], fyc[c], alpha);
#pragma unroll
        for (int l = 0; l < kQ; ++l) v[l][c] = g[l];
      }
    }
    if (MODE == 0 || MODE == 1) {
      if (active) {
#pragma unroll
        for (int l = 0; l < kQ; ++l) {
          const int slot = MODE == 1 ? opposite(l) : l;
          __stcs(reinterpret_cast<float4 *>(dst + (size_t)slot * plane + (size_t)y * pitch + x),
                 make_float4(v[l][0], v[l][1], v[l][2], v[l][3]));
        }
      }
    } else {  // AA odd phase: f*_l(x) goes to slot l at x + c_l
#pragma unroll
      for (int l = 0; l < kQ; ++l) {
        const int cxl = cx_of(l), cyl = cy_of(l);
        const int yd = cyl == 0 ? y : (cyl > 0 ? yp : ym);
        float *drow = dst + (size_t)l * plane + (size_t)yd * pitch;
        if (cxl == 0) {
          if (active)
            __stcs(reinterpret_cast<float4 *>(drow + x),
                   make_float4(v[l][0], v[l][1], v[l][2], v[l][3]));
        } else if (cxl > 0) {
          // chunk [x, x+3] receives the cells x-1 .. x+2
          const float prev = __shfl_up_sync(0xffffffffu, v[l][3], 1);
          if (active) {
            if (lane != 0) {
              __stcs(reinterpret_cast<float4 *>(drow + x),
                     make_float4(prev, v[l][0], v[l][1], v[l][2]));
            } else {
              drow[x + 1] = v[l][0];
              drow[x + 2] = v[l][1];
              drow[x + 3] = v[l][2];
            }
            if (last) drow[xnext] = v[l][3];
          }
        } else {
          // chunk [x, x+3] receives the cells x+1 .. x+4
          const float next = __shfl_down_sync(0xffffffffu, v[l][0], 1);
          if (active) {
            if (!last) {
              __stcs(reinterpret_cast<float4 *>(drow + x),
                     make_float4(v[l][1], v[l][2], v[l][3], next));
            } else {
              drow[x] = v[l][1];
              drow[x + 1] = v[l][2];
              drow[x + 2] = v[l][3];
            }
            if (lane == 0) drow[xprev] = v[l][0];
          }
        }
      }
    }
  }
}

template <int ROWS, int MODE, int PF, bool SNAP = false>
__global__ void __launch_bounds__(256, PF == 1 || PF == 2 ? 3 : (PF == 3 || SNAP ? 2 : 1)) k_step_f32_vec(const Member *__restrict__ members,
                                                      const Tile *__restrict__ tiles,
                                                      int ntiles, int cur, int flip, int snap_slot) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // flip: the tiles in reverse order, so that a step starts where the
    // previous one ended (those populations are still in L2)
    step_tile<ROWS, MODE, PF, SNAP>(members, tiles[flip ? ntiles - 1 - t : t], cur, snap_slot);
  }
}

template <int ROWS, int PF, bool SNAP = false>
static void launch_vec_rows(const Member *d_members, const Tile *d_tiles, int ntiles, int state,
                            int flip, int grid, dim3 block, cudaStream_t s, int slot = -1) {
  if (state < 2)
    k_step_f32_vec<ROWS, 0, PF, SNAP><<<grid, block, 0, s>>>(d_members, d_tiles, ntiles, state,
                                                             flip, slot);
  else if (state == 2)
    k_step_f32_vec<ROWS, 1, PF, SNAP><<<grid, block, 0, s>>>(d_members, d_tiles, ntiles, state,
                                                             flip, slot);
  else
    k_step_f32_vec<ROWS, 2, PF, SNAP><<<grid, block, 0, s>>>(d_members, d_tiles, ntiles, state,
                                                             flip, slot);
}

// pf: 0 no member with force kind 2 or a variable viscosity; 1 force kind 2
// with the BGK collision only; 2 variable-viscosity collisions (any force);
// 3 some member with the entropic collision (any other collision, any force)
template <int ROWS>
static void launch_vec_rows(const Member *d_members, const Tile *d_tiles, int ntiles, int state,
                            int flip, int grid, dim3 block, int pf, cudaStream_t s) {
  if (pf == 3)
    launch_vec_rows<ROWS, 3>(d_members, d_tiles, ntiles, state, flip, grid, block, s);
  else if (pf == 2)
    launch_vec_rows<ROWS, 2>(d_members, d_tiles, ntiles, state, flip, grid, block, s);
  else if (pf == 1)
    launch_vec_rows<ROWS, 1>(d_members, d_tiles, ntiles, state, flip, grid, block, s);
  else
    launch_vec_rows<ROWS, 0>(d_members, d_tiles, ntiles, state, flip, grid, block, s);
}

cudaError_t launch_step_f32_vec(const Member *d_members, const Tile *d_tiles, int ntiles,
                                int state, int flip, const LaunchCfg &lc, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  dim3 block(32, lc.block_warps_y);
  int grid = lc.grid_ctas > 0 ? (lc.grid_ctas < ntiles ? lc.grid_ctas : ntiles) : ntiles;
  switch (lc.rows_per_warp) {
    case 1: launch_vec_rows<1>(d_members, d_tiles, ntiles, state, flip, grid, block, lc.paper_force, s); break;
    case 2: launch_vec_rows<2>(d_members, d_tiles, ntiles, state, flip, grid, block, lc.paper_force, s); break;
    case 4: launch_vec_rows<4>(d_members, d_tiles, ntiles, state, flip, grid, block, lc.paper_force, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// One step with the snapshot of the state it reads recorded into ring slot
// `slot` (members without the paper forcing or a variable viscosity only).
cudaError_t launch_step_f32_vec_snap(const Member *d_members, const Tile *d_tiles, int ntiles,
                                     int state, int flip, const LaunchCfg &lc, int slot,
                                     cudaStream_t s) {
  if (ntiles <= 0 || lc.paper_force != 0 || slot < 0 || slot > 2) return cudaErrorInvalidValue;
  dim3 block(32, lc.block_warps_y);
  int grid = lc.grid_ctas > 0 ? (lc.grid_ctas < ntiles ? lc.grid_ctas : ntiles) : ntiles;
  switch (lc.rows_per_warp) {
    case 1: launch_vec_rows<1, 0, true>(d_members, d_tiles, ntiles, state, flip, grid, block, s, slot); break;
    case 2: launch_vec_rows<2, 0, true>(d_members, d_tiles, ntiles, state, flip, grid, block, s, slot); break;
    case 4: launch_vec_rows<4, 0, true>(d_members, d_tiles, ntiles, state, flip, grid, block, s, slot); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// General kernel: one cell per thread, any nx (FP32 deviation or FP64), any
// storage state.
// ---------------------------------------------------------------------------

// One cell (x, y) of one step of member M from storage state `state`.
// L2ONLY loads the populations past L1 (ld.global.cg): the persistent
// kernel below reads, at each step, values other SMs wrote at the previous
// one, which a stale L1 line of this SM could otherwise shadow.  The
// arithmetic is the same either way.  rec (optional): the public state
// before the step, FP64 [9][ny][nx], as k_get_pop writes it.
template <typename T, bool L2ONLY>
__device__ __forceinline__ void step_cell(const Member &M, int state, int x, int y,
                                          double *rec = nullptr) {
  const T *src = static_cast<const T *>(state_buffer(M, state));
  T *dst = static_cast<T *>(state < 2 ? M.pop[state ^ 1] : M.pop[0]);
  T fx = static_cast<const T *>(M.fx_tab)[y];
  T fy = static_cast<const T *>(M.fy_tab)[x];
  if (M.force_kind == 2) {  // shell force table + damping of eq. (16)
    const T *ft = static_cast<const T *>(M.ft_tab) + (size_t)y * M.pitch + x;
    T rx, ry;
    if constexpr (sizeof(T) == 4)
      damping_at<T, float>(M.damp_f, static_cast<const T *>(M.trig), M.nx, M.ny, x, y, rx, ry);
    else
      damping_at<T, double>(M.damp, static_cast<const T *>(M.trig), M.nx, M.ny, x, y, rx, ry);
    fx = ft[0] + rx;
    fy = ft[M.plane] + ry;
  }
  T f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const T *a = src + pub_index(M, state, l, x, y);
    if constexpr (L2ONLY)
      f[l] = __ldcg(a);
    else
      f[l] = *a;
  }
  if (rec) {
    const size_t N = (size_t)M.nx * M.ny;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      double v = (double)f[l];
      if (sizeof(T) == 4) v += w_of(l) * M.rho0;
      rec[(size_t)l * N + (size_t)y * M.nx + x] = v;
    }
  }
  if (M.collision == 3) {
    if constexpr (sizeof(T) == 4)
      collide_elbm<float>(f, M.rho0_f, M.tau_f, fx, fy, M.alpha_f);
    else
      collide_elbm<double>(f, 0.0, M.tau, fx, fy, M.alpha);
  } else if constexpr (sizeof(T) == 4) {
    collide_f32<true>(f, M.rho0_f, M.omega_f, fx, fy, M.alpha_f, M.collision, M.tau_f, M.Cs_f);
  } else {
    collide_f64(f, M.omega, fx, fy, M.alpha, M.collision, M.tau, M.Cs);
  }
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    size_t o;
    if (state < 2) {
      o = (size_t)l * M.plane + (size_t)y * M.pitch + x;
    } else if (state == 2) {
      o = (size_t)opposite(l) * M.plane + (size_t)y * M.pitch + x;
    } else {
      const int xd = wrap1(x + cx_of(l), M.nx), yd = wrap1(y + cy_of(l), M.ny);
      o = (size_t)l * M.plane + (size_t)yd * M.pitch + xd;
    }
    dst[o] = f[l];
  }
}

template <typename T>
__global__ void k_step_scalar(const Member *__restrict__ members, int member, int state,
                              double *rec) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  step_cell<T, false>(M, state, x, y, rec);
}

// ---------------------------------------------------------------------------
// Small grids: every step of a run in one cooperative launch.  A grid of a
// few thousand cells cannot fill the GPU, so a launch per step costs more in
// launch latency than in work.  Here one cooperative kernel (all CTAs
// co-resident, checked at launch) runs nsteps steps, with a grid-wide
// barrier between steps; each thread owns fixed cells and does exactly the
// general kernel's arithmetic (step_cell), so results are bit-identical.
// The barrier waits are bounded: past the limit a CTA sets the error word
// and returns, and the host reports it (LBM_ERR_TIMEOUT).
// ---------------------------------------------------------------------------

constexpr long long kBarrierSpinLimit = 1LL << 20;  // polls of ~0.5-1 us: about a second at most

// Grid-wide barrier on a monotonic arrival counter: the k-th barrier (k =
// 1, 2, ...) completes when the counter reaches k * nblocks.  Thread 0 of
// each CTA arrives with a release add (its CTA's writes, gathered by the
// __syncthreads before, become visible first) and polls with acquire loads;
// no reset, no second word.  Returns false if this CTA gave up (error word
// set by it or by another CTA).
__device__ __forceinline__ bool grid_barrier(GridSync gs, unsigned nblocks, unsigned &target) {
  __shared__ int s_ok;
  __syncthreads();
  target += nblocks;
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned v;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(v) : "l"(gs.count) : "memory");
    long long spins = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(gs.count) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((++spins & 255) == 0 &&
          (*(volatile int *)gs.err != 0 || spins > kBarrierSpinLimit)) {
        atomicExch(gs.err, 1);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kPersistThreads)
    k_step_scalar_persistent(const Member *__restrict__ members, int member, int state,
                             int nsteps, GridSync gs) {
  const Member &M = members[member];
  const int N = M.nx * M.ny;
  unsigned target = 0;
  for (int n = 0; n < nsteps; ++n) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
      step_cell<T, true>(M, state, c % M.nx, c / M.nx);
    state ^= 1;  // 0 <-> 1 (double buffer), 2 <-> 3 (AA phases)
    if (n + 1 < nsteps && !grid_barrier(gs, gridDim.x, target)) return;
  }
}

// The general kernel for several members in one launch: blockIdx.z picks
// the member from the list (grid sized for the largest; the others' surplus
// CTAs return at once), so a step of many general-kernel members (the
// entropic collision, FP64 ensembles, nx % 4 != 0) fills the GPU without a
// partial wave per member.
template <typename T>
__global__ void k_step_scalar_multi(const Member *__restrict__ members, InitList list,
                                    int state) {
  const Member &M = members[list.m[blockIdx.z]];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  step_cell<T, false>(M, state, x, y);
}

static dim3 grid2d(int nx, int ny, dim3 b) {
  return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y);
}

// CTAs for a persistent run of an N-cell member: one 32-thread CTA per 32
// cells up to one per SM, never more than can be co-resident (0 if the
// device cannot launch cooperatively).
int persistent_ctas(int precision, long long ncells) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e = precision == 32
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_scalar_persistent<float>,
                                                      kPersistThreads, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_scalar_persistent<double>,
                                                      kPersistThreads, 0);
  if (e != cudaSuccess || per_sm < 1) return 0;
  long long want = (ncells + kPersistThreads - 1) / kPersistThreads;
  if (want > sms) want = sms;
  return (int)want;
}

// The barrier alone, for the failure-detection test: `rounds` grid barriers
// over `ctas` CTAs, of which CTA `withhold` (if >= 0) never arrives, so the
// others exhaust their bounded wait, set the error word and return.
__device__ unsigned g_barrier_probe_words[4];

__global__ void k_barrier_probe(int rounds, int withhold, GridSync gs) {
  if ((int)blockIdx.x == withhold) return;
  unsigned target = 0;
  for (int r = 0; r < rounds; ++r)
    if (!grid_barrier(gs, gridDim.x, target)) return;
}

cudaError_t barrier_probe(int ctas, int rounds, int withhold, cudaStream_t s, int *gave_up) {
  unsigned *w = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void **)&w, g_barrier_probe_words);
  if (e != cudaSuccess) return e;
  GridSync gs{w, w + 1, reinterpret_cast<int *>(w + 2)};
  if ((e = cudaMemsetAsync(w, 0, 4 * sizeof(unsigned), s)) != cudaSuccess) return e;
  void *args[] = {(void *)&rounds, (void *)&withhold, (void *)&gs};
  e = cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(ctas),
                                  dim3(kPersistThreads), args, 0, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(gave_up, gs.err, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  return cudaStreamSynchronize(s);
}

cudaError_t launch_step_scalar_persistent(int precision, const Member *d_members, int member,
                                          int state, int nsteps, int ctas, GridSync gs,
                                          cudaStream_t s) {
  if (ctas < 1 || nsteps < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(gs.count, 0, 3 * sizeof(unsigned), s);  // count, gen, err
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&d_members, (void *)&member, (void *)&state, (void *)&nsteps,
                  (void *)&gs};
  if (precision == 32)
    return cudaLaunchCooperativeKernel((const void *)k_step_scalar_persistent<float>, dim3(ctas),
                                       dim3(kPersistThreads), args, 0, s);
  return cudaLaunchCooperativeKernel((const void *)k_step_scalar_persistent<double>, dim3(ctas),
                                     dim3(kPersistThreads), args, 0, s);
}

cudaError_t launch_step_scalar_batch(int precision, const Member *d_members, const int *members,
                                     int n, int nx_max, int ny_max, int state, cudaStream_t s) {
  const dim3 b = (long long)nx_max * ny_max < (1LL << 15) ? dim3(32, 2) : dim3(64, 4);
  for (int i0 = 0; i0 < n; i0 += InitList::kMax) {
    InitList list;
    list.n = n - i0 < InitList::kMax ? n - i0 : InitList::kMax;
    for (int i = 0; i < list.n; ++i) list.m[i] = members[i0 + i];
    dim3 g = grid2d(nx_max, ny_max, b);
    g.z = list.n;
    if (precision == 32)
      k_step_scalar_multi<float><<<g, b, 0, s>>>(d_members, list, state);
    else
      k_step_scalar_multi<double><<<g, b, 0, s>>>(d_members, list, state);
  }
  return cudaGetLastError();
}

cudaError_t launch_step_scalar(int precision, const Member *d_members, int member, int nx,
                               int ny, int state, cudaStream_t s, double *rec) {
  // one thread per cell; grids below 2^17 cells get 64-thread CTAs, so that
  // their FP64 arithmetic (slow on this part) spreads evenly over the SMs
  // (256^2 FP64: 16.9 against 18.2 us per step with 256-thread CTAs in 1.7
  // waves; no difference from 384^2 up)
  const dim3 b = (long long)nx * ny < (1LL << 17) ? dim3(32, 2) : dim3(64, 4);
  if (precision == 32)
    k_step_scalar<float><<<grid2d(nx, ny, b), b, 0, s>>>(d_members, member, state, rec);
  else
    k_step_scalar<double><<<grid2d(nx, ny, b), b, 0, s>>>(d_members, member, state, rec);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State conversion: init from (rho, u), public populations in and out,
// moment snapshots and the divergence flag.  All address the public
// population f_l(x, n) through pub_index.
// ---------------------------------------------------------------------------

// f(x, 0) = f_eq(rho(x), u(x)) (eq. 2) for the members of `list`
// (blockIdx.z = entry), each from its own fields at rho + entry * N etc.
// FP32 storage: the deviation t_l (rho - rho0 + rho poly) in FP32 arithmetic
// from rho - rho0 formed in FP64 (GB300 runs FP64 arithmetic and
// conversions on a slow pipe); FP64 storage: FP64 throughout.
template <typename T>
__global__ void k_init(const Member *__restrict__ members, InitList list, const double *rho,
                       const double *ux, const double *uy, int state) {
  const Member &M = members[list.m[blockIdx.z]];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  T *dst = static_cast<T *>(state_buffer(M, state));
  const size_t N = (size_t)M.nx * M.ny;
  const size_t c = (size_t)blockIdx.z * N + (size_t)y * M.nx + x;
  if constexpr (sizeof(T) == 4) {
    const float dr = (float)(rho[c] - M.rho0), r = (float)rho[c];
    const float u = (float)ux[c], v = (float)uy[c], uu = u * u + v * v;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const float cu = (float)cx_of(l) * u + (float)cy_of(l) * v;
      const float poly = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
      dst[pub_index(M, state, l, x, y)] = (float)w_of(l) * (dr + r * poly);
    }
  } else {
    const double r = rho[c], u = ux[c], v = uy[c];
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const double cu = cx_of(l) * u + cy_of(l) * v;
      const double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * (u * u + v * v);
      dst[pub_index(M, state, l, x, y)] = (T)(w_of(l) * r * (1.0 + poly));
    }
  }
}

template <typename T>
__global__ void k_get_pop(const Member *__restrict__ members, int member, int state, double *f) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(state_buffer(M, state));
  const size_t N = (size_t)M.nx * M.ny;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    double v = (double)src[pub_index(M, state, l, x, y)];
    if (sizeof(T) == 4) v += w_of(l) * M.rho0;
    f[(size_t)l * N + (size_t)y * M.nx + x] = v;
  }
}

template <typename T>
__global__ void k_set_pop(const Member *__restrict__ members, int member, int state,
                          const double *f) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  T *dst = static_cast<T *>(state_buffer(M, state));
  const size_t N = (size_t)M.nx * M.ny;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    double v = f[(size_t)l * N + (size_t)y * M.nx + x];
    if (sizeof(T) == 4) v -= w_of(l) * M.rho0;
    dst[pub_index(M, state, l, x, y)] = (T)v;
  }
}

// (rho, j_x, j_y) of the pre-collision state, FP64, into d[3][ny*nx]; with a
// variable-viscosity collision also the local viscosity as d[3][ny*nx].
template <typename T>
__global__ void k_snapshot(const Member *__restrict__ members, int member, int state,
                           double *d) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(state_buffer(M, state));
  T f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) f[l] = src[pub_index(M, state, l, x, y)];
  double r, jx, jy;
  pub_moments<T>(f, M.rho0, r, jx, jy);
  const size_t N = (size_t)M.nx * M.ny, c = (size_t)y * M.nx + x;
  d[c] = r;
  d[N + c] = jx;
  d[2 * N + c] = jy;
  if (M.collision != 0) {  // local viscosity as a fourth field
    double t;
    if (M.collision == 3) {
      if constexpr (sizeof(T) == 4)
        t = (double)elbm_tau<float>(f, M.rho0_f, M.tau_f);
      else
        t = elbm_tau<double>(f, 0.0, M.tau);
    } else if constexpr (sizeof(T) == 4) {
      float drho, rho, jxf, jyf, ir, ux, uy;
      moments_f32(f, M.rho0_f, drho, rho, jxf, jyf, ir, ux, uy);
      t = (double)local_tau_f32(f, drho, rho, ux, uy, M.tau_f, M.collision, M.Cs_f);
    } else {
      double rho, ux, uy;
      moments_f64(f, rho, ux, uy);
      t = local_tau_f64(f, rho, ux, uy, M.tau, M.collision, M.Cs);
    }
    d[3 * N + c] = (t - 0.5) / 3.0;
  }
}

// The snapshot ring entry of every member at once (blockIdx.z = member):
// (rho, j_x, j_y) of the pre-collision state into ring slot `slot` of
// M.snap.  FP64 storage: [3][N] doubles.  FP32 deviation storage: [3][2][N]
// floats, the compensated pairs (hi, lo) of rho - rho0, j_x, j_y.
template <typename T>
__global__ void k_snapshot_ring(const Member *__restrict__ members, int state, int slot) {
  const Member &M = members[blockIdx.z];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(state_buffer(M, state));
  T f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) f[l] = src[pub_index(M, state, l, x, y)];
  const size_t N = (size_t)M.nx * M.ny, c = (size_t)y * M.nx + x;
  if constexpr (sizeof(T) == 4) {
    const int one[kQ] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    const float ax[6] = {f[1], f[5], f[8], f[3], f[6], f[7]};
    const float ay[6] = {f[2], f[5], f[6], f[4], f[7], f[8]};
    const int sgn[6] = {1, 1, 1, -1, -1, -1};
    float hi[3], lo[3];
    csum_pair(f, one, kQ, hi[0], lo[0]);
    csum_pair(ax, sgn, 6, hi[1], lo[1]);
    csum_pair(ay, sgn, 6, hi[2], lo[2]);
    float *d = reinterpret_cast<float *>(M.snap) + (size_t)slot * 6 * N;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      d[(size_t)(2 * q) * N + c] = hi[q];
      d[(size_t)(2 * q + 1) * N + c] = lo[q];
    }
    if (M.collision != 0) {  // the local viscosity the step from this state uses
      float t;
      if (M.collision == 3) {
        t = elbm_tau<float>(f, M.rho0_f, M.tau_f);
      } else {
        float drho, rho, jx, jy, ir, ux, uy;
        moments_f32(f, M.rho0_f, drho, rho, jx, jy, ir, ux, uy);
        t = local_tau_f32(f, drho, rho, ux, uy, M.tau_f, M.collision, M.Cs_f);
      }
      static_cast<float *>(M.nu_ring)[(size_t)slot * N + c] = (t - 0.5f) * (1.0f / 3.0f);
    }
  } else {
    double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      r += f[l];
      if (cx_of(l) != 0) jx += cx_of(l) * f[l];
      if (cy_of(l) != 0) jy += cy_of(l) * f[l];
    }
    double *d = M.snap + (size_t)slot * 3 * N;
    d[c] = r;
    d[N + c] = jx;
    d[2 * N + c] = jy;
    if (M.collision != 0) {
      double t;
      if (M.collision == 3) {
        t = elbm_tau<double>(f, 0.0, M.tau);
      } else {
        double rho, ux, uy;
        moments_f64(f, rho, ux, uy);
        t = local_tau_f64(f, rho, ux, uy, M.tau, M.collision, M.Cs);
      }
      static_cast<double *>(M.nu_ring)[(size_t)slot * N + c] = (t - 0.5) / 3.0;
    }
  }
}

// The member's last projection CTA to finish (a counter in
// Member::proj_count; the caller wrote its partials and fenced) reduces the
// nblk CTA partials in a fixed order into the damping coefficients and, for
// the running step of FP32 storage, the per-row factors.  Every thread of
// the CTA calls it (256 threads: tid, lane, wid of the CTA).
__device__ void project_finalize(const Member &M, int nblk, int slot, int tid, int lane, int wid) {
  const int nx = M.nx, ny = M.ny;
  __shared__ int is_last;
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(M.proj_count, 1u) == (unsigned)(nblk - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // last CTA: one warp per value, two fixed-order chains and a shuffle tree
  __shared__ double coef[kDamp];
  const int nthreads = blockDim.x * blockDim.y, nwarps = nthreads >> 5;
  for (int q = wid; q < kDamp; q += nwarps) {
    double a0 = 0.0, a1 = 0.0;
    int b = lane;
    for (; b + 32 < nblk; b += 64) {
      a0 += __ldcg(M.proj_part + (size_t)b * kDamp + q);
      a1 += __ldcg(M.proj_part + (size_t)(b + 32) * kDamp + q);
    }
    if (b < nblk) a0 += __ldcg(M.proj_part + (size_t)b * kDamp + q);
    double a = a0 + a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) {
      const double c = -2.0 * M.FR0 * a / ((double)nx * (double)ny);
      coef[q] = c;
      if (slot < 0) {
        M.damp[q] = c;
        M.damp_f[q] = (float)c;
      } else {
        M.damp_ring[slot * kDamp + q] = c;
      }
    }
  }
  if (tid == 0) *M.proj_count = 0u;  // ready for the next launch
  if (slot >= 0 || M.damp_rows == nullptr) return;
  __syncthreads();
  // per-row factors of the FP32 step in FP32 arithmetic (they are stored as
  // FP32; FP64 arithmetic here is the slow pipe at the end of the kernel)
  __shared__ float coef_f[kDamp];
  if (tid < kDamp) coef_f[tid] = (float)coef[tid];
  __syncthreads();
  const float *tyf = static_cast<const float *>(M.trig) + 4 * (size_t)nx;
  for (int y = tid; y < ny; y += nthreads) {
    const float cy = tyf[y], sy = tyf[ny + y], c2y = tyf[2 * ny + y], s2y = tyf[3 * ny + y];
    float *row = M.damp_rows + 6 * (size_t)y;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float *d = coef_f + 12 * k;
      row[3 * k] = d[0] + (d[4] + d[6]) * cy + (d[5] - d[7]) * sy;
      row[3 * k + 1] = d[1] + (d[5] + d[7]) * cy - (d[4] - d[6]) * sy;
      row[3 * k + 2] = d[2] * cy + d[3] * sy + d[10] * c2y + d[11] * s2y;
    }
  }
}

// Projection for the damping of eq. (16): each CTA (64 x 64 cells of member
// blockIdx.z; every thread 16 rows, 4 apart) sums u_c cos(theta_m) and
// u_c sin(theta_m) over its cells, u = j / rho the bare velocity of the
// state in storage `state`, in the order of kDamp, and stores the sums
// (FP64) at its slot of Member::proj_part.  The member's last CTA to finish
// (a counter in Member::proj_count) reduces the slots in a fixed order into
// the coefficients: slot < 0 into Member::damp / damp_f and, for FP32
// storage, the per-row factors P(y) cos(a_x) + Q(y) sin(a_x) + R(y) of
// damping_at in Member::damp_rows[y] = (P, Q, R) of x, then of y; slot
// 0..2 into that ring slot of Member::damp_ring.
constexpr int kProjRows = 16;
template <typename T>
__global__ void __launch_bounds__(256) k_project(const Member *__restrict__ members, int state,
                                                 int slot) {
  const Member &M = members[blockIdx.z];
  if (M.force_kind != 2) return;
  if ((int)(blockIdx.x * 64) >= M.nx || (int)(blockIdx.y * 4 * kProjRows) >= M.ny) return;
  const int nx = M.nx, ny = M.ny;
  const int x = blockIdx.x * 64 + threadIdx.x;
  T acc[kDamp];
#pragma unroll
  for (int q = 0; q < kDamp; ++q) acc[q] = T(0);
  const T *src = static_cast<const T *>(state_buffer(M, state));
  const T *tr = static_cast<const T *>(M.trig);
  T cx = 0, sx = 0, c2x = 0, s2x = 0;
  if (x < nx) {
    cx = tr[x];
    sx = tr[nx + x];
    c2x = tr[2 * nx + x];
    s2x = tr[3 * nx + x];
  }
#pragma unroll 4
  for (int r = 0; r < kProjRows; ++r) {
    const int y = blockIdx.y * 4 * kProjRows + r * 4 + threadIdx.y;
    if (x >= nx || y >= ny) continue;
    T f[kQ];
#pragma unroll
    for (int l = 0; l < kQ; ++l) f[l] = src[pub_index(M, state, l, x, y)];
    T rho = sizeof(T) == 4 ? (T)M.rho0_f : T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      rho += f[l];
      if (cx_of(l) != 0) jx += (T)cx_of(l) * f[l];
      if (cy_of(l) != 0) jy += (T)cy_of(l) * f[l];
    }
    const T ir = T(1) / rho;
    const T u[2] = {jx * ir, jy * ir};
    const T cy = tr[4 * nx + y], sy = tr[4 * nx + ny + y];
    const T c2y = tr[4 * nx + 2 * ny + y], s2y = tr[4 * nx + 3 * ny + y];
    const T cm[6] = {cx, cy, cx * cy - sx * sy, cx * cy + sx * sy, c2x, c2y};
    const T sm[6] = {sx, sy, sx * cy + cx * sy, sx * cy - cx * sy, s2x, s2y};
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        acc[12 * k + 2 * m] += u[k] * cm[m];
        acc[12 * k + 2 * m + 1] += u[k] * sm[m];
      }
  }
  // CTA sums in T, widened to FP64 once per CTA and value: a per-warp
  // widening would put 24 conversions per warp on GB300's slow FP64 pipe
  __shared__ T sh[kDamp][8];
  const int tid = threadIdx.y * 64 + threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int q = 0; q < kDamp; ++q) {
    T a = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = a;
  }
  __syncthreads();
  const int nblk = ((nx + 63) / 64) * ((ny + 4 * kProjRows - 1) / (4 * kProjRows));
  if (tid < kDamp) {
    T a = sh[tid][0];
    for (int w = 1; w < 8; ++w) a += sh[tid][w];
    const int blk = blockIdx.y * ((nx + 63) / 64) + blockIdx.x;
    M.proj_part[(size_t)blk * kDamp + tid] = (double)a;
    __threadfence();
  }
  project_finalize(M, nblk, slot, tid, lane, wid);
}

// FP32 projection with 4 consecutive cells per lane (every kind-2 member
// with nx % 4 == 0): CTA (32, 8), a warp per 128-cell row segment, each
// thread kProj4Rows rows 8 apart, so a CTA covers 128 x 8 kProj4Rows cells.
// The populations of the state are pulled as in k_step_f32_vec (MODE 0:
// double buffer `state`, 1: AA even, 2: AA odd): one float4 per population
// and lane, the x-shift by shuffles.  Same sums per cell as k_project.
// One row's contribution to the 24 damping-mode sums: rho, jx, jy are the
// moments (rho with rho0 added) of four consecutive cells of row y (the
// lane's cells), cx..s2x their x trig factors.
__device__ __forceinline__ void proj_row_accumulate(const Member &M, const float (&rho)[4],
                                                    const float (&jx)[4], const float (&jy)[4],
                                                    const float (&cx)[4], const float (&sx)[4],
                                                    const float (&c2x)[4], const float (&s2x)[4],
                                                    int y, float (&acc)[kDamp]) {
  const int nx = M.nx, ny = M.ny;
  const float *tr = static_cast<const float *>(M.trig);
  const float cy = tr[4 * nx + y], sy = tr[4 * nx + ny + y];
  const float c2y = tr[4 * nx + 2 * ny + y], s2y = tr[4 * nx + 3 * ny + y];
  // separable in x and y: the lane's sums of u (1, cos x, sin x, cos 2x,
  // sin 2x) over its four cells, folded into the mode sums with the row's
  // y factors (cos(x +- y) = cx cy -+ sx sy, sin(x +- y) = sx cy +- cx sy)
  float R[2][5];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int q = 0; q < 5; ++q) R[k][q] = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // approximate reciprocal (2 ulp): u only enters the damping's mode sums,
    // whose force is F^R_0 ~ 1e-5 times them
    const float ir = __fdividef(1.0f, rho[i]);
    const float u[2] = {jx[i] * ir, jy[i] * ir};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      R[k][0] += u[k];
      R[k][1] += u[k] * cx[i];
      R[k][2] += u[k] * sx[i];
      R[k][3] += u[k] * c2x[i];
      R[k][4] += u[k] * s2x[i];
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float *a = acc + 12 * k;
    a[0] += R[k][1];                       // cos x
    a[1] += R[k][2];                       // sin x
    a[2] += R[k][0] * cy;                  // cos y
    a[3] += R[k][0] * sy;                  // sin y
    a[4] += R[k][1] * cy - R[k][2] * sy;   // cos(x + y)
    a[5] += R[k][2] * cy + R[k][1] * sy;   // sin(x + y)
    a[6] += R[k][1] * cy + R[k][2] * sy;   // cos(x - y)
    a[7] += R[k][2] * cy - R[k][1] * sy;   // sin(x - y)
    a[8] += R[k][3];                       // cos 2x
    a[9] += R[k][4];                       // sin 2x
    a[10] += R[k][0] * c2y;                // cos 2y
    a[11] += R[k][0] * s2y;                // sin 2y
  }
}

// The loads of one row of k_project4's pull (MODE 0: double buffer, 1: AA
// even, 2: AA odd): one float4 per population and lane (o), and e[l] the
// cell beyond the lane's chunk that the x-shift needs where no neighbouring
// lane holds it (lane 0 for c_x > 0, the last active lane for c_x < 0).
template <int MODE>
__device__ __forceinline__ void proj4_load(const Member &M, const float *src, int y, int x,
                                           int xprev, int xnext, bool active, bool last,
                                           int lane, float4 (&o)[kQ], float (&e)[kQ]) {
  const int ny = M.ny, pitch = M.pitch;
  const size_t plane = M.plane;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y + 1 == ny ? 0 : y + 1;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int cxl = MODE == 1 ? 0 : cx_of(l), cyl = cy_of(l);
    const int sl = MODE == 2 ? opposite(l) : l;
    const int ys = MODE == 1 || cyl == 0 ? y : (cyl > 0 ? ym : yp);  // from y - c_y
    const float *row = src + (size_t)sl * plane + (size_t)ys * pitch;
    o[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    e[l] = 0.f;
    if (active) o[l] = __ldg(reinterpret_cast<const float4 *>(row + x));
    if (cxl > 0 && active && lane == 0) e[l] = __ldg(row + xprev);
    if (cxl < 0 && last) e[l] = __ldg(row + xnext);
  }
}

// The moments of the lane's four cells from one row's loads: the x-shift of
// the pull by shuffles, e[l] at the chunk's edge.
template <int MODE>
__device__ __forceinline__ void proj4_moments(float rho0, const float4 (&o)[kQ],
                                              const float (&e)[kQ], bool active, bool last,
                                              int lane, float (&rho)[4], float (&jx)[4],
                                              float (&jy)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    rho[i] = rho0;
    jx[i] = 0.f;
    jy[i] = 0.f;
  }
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int cxl = MODE == 1 ? 0 : cx_of(l);
    float v[4];
    if (cxl == 0) {
      v[0] = o[l].x; v[1] = o[l].y; v[2] = o[l].z; v[3] = o[l].w;
    } else if (cxl > 0) {  // from x - 1
      float prev = __shfl_up_sync(0xffffffffu, o[l].w, 1);
      if (active && lane == 0) prev = e[l];
      v[0] = prev; v[1] = o[l].x; v[2] = o[l].y; v[3] = o[l].z;
    } else {  // from x + 1
      float next = __shfl_down_sync(0xffffffffu, o[l].x, 1);
      if (last) next = e[l];
      v[0] = o[l].y; v[1] = o[l].z; v[2] = o[l].w; v[3] = next;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      rho[i] += v[i];
      if (cx_of(l) != 0) jx[i] += (float)cx_of(l) * v[i];
      if (cy_of(l) != 0) jy[i] += (float)cy_of(l) * v[i];
    }
  }
}
// Block (bx, by) of the projection of member M: cells [128 bx, 128 bx + 128)
// x [8 prow by, 8 prow (by + 1)), CTA (32, 8), prow rows per thread.
template <int MODE>
__device__ __forceinline__ void proj4_block(const Member &M, int bx, int by, int state, int slot,
                                            int prow) {
  const int nx = M.nx, ny = M.ny, lane = threadIdx.x;
  const int x = bx * 128 + 4 * lane;
  const bool active = x < nx;
  const bool last = active && (lane == 31 || x + 4 >= nx);
  const int xprev = x == 0 ? nx - 1 : x - 1, xnext = x + 4 >= nx ? 0 : x + 4;
  const float *src = static_cast<const float *>(MODE == 0 ? M.pop[state] : M.pop[0]);
  const float *tr = static_cast<const float *>(M.trig);
  float cx[4] = {0, 0, 0, 0}, sx[4] = {0, 0, 0, 0}, c2x[4] = {0, 0, 0, 0}, s2x[4] = {0, 0, 0, 0};
  if (active) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      cx[i] = tr[x + i];
      sx[i] = tr[nx + x + i];
      c2x[i] = tr[2 * nx + x + i];
      s2x[i] = tr[3 * nx + x + i];
    }
  }
  float acc[kDamp];
#pragma unroll
  for (int q = 0; q < kDamp; ++q) acc[q] = 0.f;
  // software-pipelined over the thread's rows: the loads of the next row are
  // issued before the mode sums of the current one
  float4 o[kQ];
  float e[kQ];
  const int yb = by * 8 * prow + threadIdx.y;
  if (yb < ny) proj4_load<MODE>(M, src, yb, x, xprev, xnext, active, last, lane, o, e);
#pragma unroll 1
  for (int r = 0; r < prow; ++r) {
    const int y = yb + 8 * r;
    if (y >= ny) break;  // whole warps
    float rho[4], jx[4], jy[4];
    proj4_moments<MODE>(M.rho0_f, o, e, active, last, lane, rho, jx, jy);
    if (r + 1 < prow && y + 8 < ny)
      proj4_load<MODE>(M, src, y + 8, x, xprev, xnext, active, last, lane, o, e);
    if (active) proj_row_accumulate(M, rho, jx, jy, cx, sx, c2x, s2x, y, acc);
  }
  __shared__ float sh[kDamp][8];
  const int tid = threadIdx.y * 32 + threadIdx.x, wid = threadIdx.y;
#pragma unroll
  for (int q = 0; q < kDamp; ++q) {
    float a = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = a;
  }
  __syncthreads();
  const int gx = (nx + 127) / 128;
  const int nblk = gx * ((ny + 8 * prow - 1) / (8 * prow));
  if (tid < kDamp) {
    float a = sh[tid][0];
    for (int w = 1; w < 8; ++w) a += sh[tid][w];
    M.proj_part[(size_t)(by * gx + bx) * kDamp + tid] = (double)a;
    __threadfence();
  }
  project_finalize(M, nblk, slot, tid, lane, wid);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_project4(const Member *__restrict__ members, int state,
                                                  int slot, int prow) {
  const Member &M = members[blockIdx.z];
  if (M.force_kind != 2) return;
  if ((int)(blockIdx.x * 128) >= M.nx || (int)(blockIdx.y * 8 * prow) >= M.ny) return;
  proj4_block<MODE>(M, blockIdx.x, blockIdx.y, state, slot, prow);
}


// The snapshot-ring entry of FP32 members with nx % 4 == 0 and a constant
// viscosity, four cells per lane: CTA (32, 8), a warp per 128-cell row
// segment, kSnap4Rows rows per thread 8 apart; the state pulled as in
// k_step_f32_vec (MODE 0: double buffer `state`, 1: AA even, 2: AA odd) and
// the same compensated pairs as k_snapshot_ring and the recording step.
constexpr int kSnap4Rows = 4;
template <int MODE>
__global__ void __launch_bounds__(256) k_snapshot4(const Member *__restrict__ members, int state,
                                                   int slot) {
  const Member &M = members[blockIdx.z];
  if ((int)(blockIdx.x * 128) >= M.nx || (int)(blockIdx.y * 8 * kSnap4Rows) >= M.ny) return;
  const int nx = M.nx, ny = M.ny, pitch = M.pitch, lane = threadIdx.x;
  const size_t plane = M.plane, N = (size_t)nx * ny;
  const int x = blockIdx.x * 128 + 4 * lane;
  const bool active = x < nx;
  const bool last = active && (lane == 31 || x + 4 >= nx);
  const int xprev = x == 0 ? nx - 1 : x - 1, xnext = x + 4 >= nx ? 0 : x + 4;
  const float *src = static_cast<const float *>(MODE == 0 ? M.pop[state] : M.pop[0]);
  float *ring = reinterpret_cast<float *>(M.snap) + (size_t)slot * 6 * N;
#pragma unroll 1
  for (int r = 0; r < kSnap4Rows; ++r) {
    const int y = blockIdx.y * 8 * kSnap4Rows + r * 8 + threadIdx.y;
    if (y >= ny) break;  // whole warps
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y + 1 == ny ? 0 : y + 1;
    float v[kQ][4];
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      const int cxl = cx_of(l), cyl = cy_of(l);
      if (MODE == 1) {  // own cell, own slot
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active)
          o = __ldg(reinterpret_cast<const float4 *>(src + (size_t)l * plane + (size_t)y * pitch + x));
        v[l][0] = o.x; v[l][1] = o.y; v[l][2] = o.z; v[l][3] = o.w;
        continue;
      }
      const int sl = MODE == 2 ? opposite(l) : l;
      const int ys = cyl == 0 ? y : (cyl > 0 ? ym : yp);  // from y - c_y
      const float *row = src + (size_t)sl * plane + (size_t)ys * pitch;
      float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
      if (active) o = __ldg(reinterpret_cast<const float4 *>(row + x));
      if (cxl == 0) {
        v[l][0] = o.x; v[l][1] = o.y; v[l][2] = o.z; v[l][3] = o.w;
      } else if (cxl > 0) {  // from x - 1
        float prev = __shfl_up_sync(0xffffffffu, o.w, 1);
        if (active && (lane == 0 || x == 0)) prev = __ldg(row + xprev);
        v[l][0] = prev; v[l][1] = o.x; v[l][2] = o.y; v[l][3] = o.z;
      } else {  // from x + 1
        float next = __shfl_down_sync(0xffffffffu, o.x, 1);
        if (last) next = __ldg(row + xnext);
        v[l][0] = o.y; v[l][1] = o.z; v[l][2] = o.w; v[l][3] = next;
      }
    }
    if (!active) continue;
    float hs[3][4], ls[3][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int one[kQ] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
      const int sgn[6] = {1, 1, 1, -1, -1, -1};
      float f[kQ];
#pragma unroll
      for (int l = 0; l < kQ; ++l) f[l] = v[l][c];
      const float ax[6] = {f[1], f[5], f[8], f[3], f[6], f[7]};
      const float ay[6] = {f[2], f[5], f[6], f[4], f[7], f[8]};
      csum_pair(f, one, kQ, hs[0][c], ls[0][c]);
      csum_pair(ax, sgn, 6, hs[1][c], ls[1][c]);
      csum_pair(ay, sgn, 6, hs[2][c], ls[2][c]);
    }
    float *d = ring + (size_t)y * nx + x;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      __stcs(reinterpret_cast<float4 *>(d + (size_t)(2 * q) * N),
             make_float4(hs[q][0], hs[q][1], hs[q][2], hs[q][3]));
      __stcs(reinterpret_cast<float4 *>(d + (size_t)(2 * q + 1) * N),
             make_float4(ls[q][0], ls[q][1], ls[q][2], ls[q][3]));
    }
  }
}

template <typename T>
__global__ void k_status(const Member *__restrict__ members, int member, int state) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(state_buffer(M, state));
  double r = 0.0;
  bool bad = false;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const double v = (double)src[pub_index(M, state, l, x, y)];
    bad |= !isfinite(v);
    r += v;
  }
  if (sizeof(T) == 4) r += M.rho0;
  if (bad || !(r > 0.0)) atomicOr(M.status, 1);
}

#define LBM_DISPATCH(prec, kern, ...)                                   \
  do {                                                                  \
    dim3 b(64, 4);                                                      \
    dim3 g = grid2d(nx, ny, b);                                         \
    if ((prec) == 32)                                                   \
      kern<float><<<g, b, 0, s>>>(__VA_ARGS__);                         \
    else                                                                \
      kern<double><<<g, b, 0, s>>>(__VA_ARGS__);                        \
  } while (0)

cudaError_t launch_init_fields(int precision, const Member *d_members, const int *members, int n,
                               int nx, int ny, const double *rho, const double *ux,
                               const double *uy, int state, cudaStream_t s) {
  const size_t N = (size_t)nx * ny;
  for (int i0 = 0; i0 < n; i0 += InitList::kMax) {
    InitList list;
    list.n = n - i0 < InitList::kMax ? n - i0 : InitList::kMax;
    for (int i = 0; i < list.n; ++i) list.m[i] = members[i0 + i];
    const dim3 b(64, 4);
    dim3 g = grid2d(nx, ny, b);
    g.z = list.n;
    const size_t o = (size_t)i0 * N;
    if (precision == 32)
      k_init<float><<<g, b, 0, s>>>(d_members, list, rho + o, ux + o, uy + o, state);
    else
      k_init<double><<<g, b, 0, s>>>(d_members, list, rho + o, ux + o, uy + o, state);
  }
  return cudaGetLastError();
}

cudaError_t launch_get_populations(int precision, const Member *d_members, int member,
                                   int nx, int ny, int state, double *f, cudaStream_t s) {
  LBM_DISPATCH(precision, k_get_pop, d_members, member, state, f);
  return cudaGetLastError();
}

cudaError_t launch_set_populations(int precision, const Member *d_members, int member,
                                   int nx, int ny, int state, const double *f, cudaStream_t s) {
  LBM_DISPATCH(precision, k_set_pop, d_members, member, state, f);
  return cudaGetLastError();
}

cudaError_t launch_snapshot(int precision, const Member *d_members, int member, int nx,
                            int ny, int state, double *dst, cudaStream_t s) {
  LBM_DISPATCH(precision, k_snapshot, d_members, member, state, dst);
  return cudaGetLastError();
}

cudaError_t launch_snapshot_ring(int precision, const Member *d_members, int n_members,
                                 int nx_max, int ny_max, int state, int slot, bool quad,
                                 cudaStream_t s) {
  if (quad && precision == 32) {  // four cells per lane
    const dim3 g4((nx_max + 127) / 128, (ny_max + 8 * kSnap4Rows - 1) / (8 * kSnap4Rows),
                  n_members);
    const dim3 b4(32, 8);
    if (state < 2)
      k_snapshot4<0><<<g4, b4, 0, s>>>(d_members, state, slot);
    else if (state == 2)
      k_snapshot4<1><<<g4, b4, 0, s>>>(d_members, state, slot);
    else
      k_snapshot4<2><<<g4, b4, 0, s>>>(d_members, state, slot);
    return cudaGetLastError();
  }
  const dim3 b(64, 4);
  dim3 g = grid2d(nx_max, ny_max, b);
  g.z = n_members;
  if (precision == 32)
    k_snapshot_ring<float><<<g, b, 0, s>>>(d_members, state, slot);
  else
    k_snapshot_ring<double><<<g, b, 0, s>>>(d_members, state, slot);
  return cudaGetLastError();
}

cudaError_t launch_projection(int precision, const Member *d_members, int n_members,
                              int nx_max, int ny_max, int state, int slot, bool quad, int prow,
                              cudaStream_t s) {
  if (quad && precision == 32) {  // four cells per lane
    if (prow < 1) return cudaErrorInvalidValue;
    dim3 g((nx_max + 127) / 128, (ny_max + 8 * prow - 1) / (8 * prow), n_members);
    const dim3 b4(32, 8);
    if (state < 2)
      k_project4<0><<<g, b4, 0, s>>>(d_members, state, slot, prow);
    else if (state == 2)
      k_project4<1><<<g, b4, 0, s>>>(d_members, state, slot, prow);
    else
      k_project4<2><<<g, b4, 0, s>>>(d_members, state, slot, prow);
    return cudaGetLastError();
  }
  const dim3 b(64, 4);
  dim3 g = grid2d(nx_max, ny_max, dim3(64, 4 * kProjRows));
  g.z = n_members;
  if (precision == 32)
    k_project<float><<<g, b, 0, s>>>(d_members, state, slot);
  else
    k_project<double><<<g, b, 0, s>>>(d_members, state, slot);
  return cudaGetLastError();
}

cudaError_t launch_status(int precision, const Member *d_members, int member, int nx,
                          int ny, int state, cudaStream_t s) {
  LBM_DISPATCH(precision, k_status, d_members, member, state);
  return cudaGetLastError();
}

}  // namespace lbm
