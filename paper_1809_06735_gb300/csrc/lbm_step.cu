// D2Q9 BGK stream-collide with exact-difference forcing (eq. (1), eq. (2),
// Sec. 3 of Tauzin et al. 2018) and the kernels that move the state in and
// out of the device storage convention (see lbm_internal.cuh).
//
// Hot kernel: k_step_f32_vec, one pass per time step over every member of
// the ensemble.  Each warp owns 128 consecutive cells of one row (4 per
// lane); each of the 9 populations is fetched with one aligned 128-bit load
// per lane from the source row y - c_y, and the +-1 shift of the x-moving
// populations is done with a warp shuffle (one scalar load at each warp
// edge), so DRAM sees 9 x 16 B of coalesced reads and 9 x 16 B of writes per
// 4 cells: the algorithmic 72 B per lattice update.
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
__device__ __forceinline__ void collide_f32(float g[kQ], float rho0, float om, float Fex,
                                            float Fey, float alpha) {
  const float drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
  const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
  const float rho = rho0 + drho;
  const float ir = 1.0f / rho;
  const float ux = jx * ir, uy = jy * ir;
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

// FP64 plain form on the full populations f_l.
__device__ __forceinline__ void collide_f64(double f[kQ], double om, double Fex, double Fey,
                                            double alpha) {
  double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    rho += f[l];
    jx += cx_of(l) * f[l];
    jy += cy_of(l) * f[l];
  }
  const double ir = 1.0 / rho;
  const double ux = jx * ir, uy = jy * ir;
  const double Fx = Fex - alpha * jx, Fy = Fey - alpha * jy;
  const double dux = Fx * ir, duy = Fy * ir;
  const double usq = ux * ux + uy * uy;
  const double dsq = dux * (2.0 * ux + dux) + duy * (2.0 * uy + duy);
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const double t = w_of(l);
    const double cu = cx_of(l) * ux + cy_of(l) * uy;
    const double cd = cx_of(l) * dux + cy_of(l) * duy;
    const double feq = t * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    const double Fl = t * rho * (3.0 * cd + 4.5 * cd * (2.0 * cu + cd) - 1.5 * dsq);
    f[l] = f[l] - om * (f[l] - feq) + Fl;
  }
}

// ---------------------------------------------------------------------------
// Hot kernel: batched FP32 stream-collide, 4 cells per lane, nx % 4 == 0.
// blockDim = (32, WY); a tile is 128 x (WY * ROWS) cells of one member.
// ---------------------------------------------------------------------------

template <int ROWS>
__global__ void __launch_bounds__(256) k_step_f32_vec(const Member *__restrict__ members,
                                                      const Tile *__restrict__ tiles,
                                                      int ntiles, int cur) {
  const int lane = threadIdx.x;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const Member &M = members[tl.member];
    const int nx = M.nx, ny = M.ny, pitch = M.pitch;
    const size_t plane = M.plane;
    const float *__restrict__ src = static_cast<const float *>(M.pop[cur]);
    float *__restrict__ dst = static_cast<float *>(M.pop[cur ^ 1]);
    const float *__restrict__ fxt = static_cast<const float *>(M.fx_tab);
    const float *__restrict__ fyt = static_cast<const float *>(M.fy_tab);
    const float rho0 = M.rho0_f, om = M.omega_f, alpha = M.alpha_f;
    const int x = tl.x0 + 4 * lane;
    const bool active = x < nx;
    float4 fy4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) fy4 = *reinterpret_cast<const float4 *>(fyt + x);
    const float fy[4] = {fy4.x, fy4.y, fy4.z, fy4.w};
    const int xprev = (x == 0) ? nx - 1 : x - 1;   // source of lane 0's c_x=+1 cell
    const int xnext = (x + 4 >= nx) ? 0 : x + 4;   // source of last cell's c_x=-1

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
        const int ys = cyl == 0 ? y : (cyl > 0 ? ym : yp);  // pull from y - c_y
        const float *row = src + (size_t)l * plane + (size_t)ys * pitch;
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active) o = __ldg(reinterpret_cast<const float4 *>(row + x));
        if (cxl == 0) {
          v[l][0] = o.x; v[l][1] = o.y; v[l][2] = o.z; v[l][3] = o.w;
        } else if (cxl > 0) {  // pull from x - 1
          float prev = __shfl_up_sync(0xffffffffu, o.w, 1);
          if (active && (lane == 0 || x == 0)) prev = __ldg(row + xprev);
          v[l][0] = prev; v[l][1] = o.x; v[l][2] = o.y; v[l][3] = o.z;
        } else {  // pull from x + 1
          float next = __shfl_down_sync(0xffffffffu, o.x, 1);
          if (active && (lane == 31 || x + 4 >= nx)) next = __ldg(row + xnext);
          v[l][0] = o.y; v[l][1] = o.z; v[l][2] = o.w; v[l][3] = next;
        }
      }
      if (active) {
        const float fx = fxt[y];
        float out[kQ][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float g[kQ];
#pragma unroll
          for (int l = 0; l < kQ; ++l) g[l] = v[l][c];
          collide_f32(g, rho0, om, fx, fy[c], alpha);
#pragma unroll
          for (int l = 0; l < kQ; ++l) out[l][c] = g[l];
        }
        float *drow = dst + (size_t)y * pitch + x;
#pragma unroll
        for (int l = 0; l < kQ; ++l)
          __stcs(reinterpret_cast<float4 *>(drow + (size_t)l * plane),
                 make_float4(out[l][0], out[l][1], out[l][2], out[l][3]));
      }
    }
  }
}

cudaError_t launch_step_f32_vec(const Member *d_members, const Tile *d_tiles, int ntiles,
                                int cur, const LaunchCfg &lc, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  dim3 block(32, lc.block_warps_y);
  int grid = lc.grid_ctas > 0 ? (lc.grid_ctas < ntiles ? lc.grid_ctas : ntiles) : ntiles;
  switch (lc.rows_per_warp) {
    case 1: k_step_f32_vec<1><<<grid, block, 0, s>>>(d_members, d_tiles, ntiles, cur); break;
    case 2: k_step_f32_vec<2><<<grid, block, 0, s>>>(d_members, d_tiles, ntiles, cur); break;
    case 4: k_step_f32_vec<4><<<grid, block, 0, s>>>(d_members, d_tiles, ntiles, cur); break;
    case 8: k_step_f32_vec<8><<<grid, block, 0, s>>>(d_members, d_tiles, ntiles, cur); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// General kernel: one cell per thread, any nx (FP32 deviation or FP64).
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_step_scalar(const Member *__restrict__ members, int member, int cur) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *__restrict__ src = static_cast<const T *>(M.pop[cur]);
  T *__restrict__ dst = static_cast<T *>(M.pop[cur ^ 1]);
  const T fx = static_cast<const T *>(M.fx_tab)[y];
  const T fy = static_cast<const T *>(M.fy_tab)[x];
  T f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int xs = wrapi(x - cx_of(l), M.nx), ys = wrapi(y - cy_of(l), M.ny);
    f[l] = src[(size_t)l * M.plane + (size_t)ys * M.pitch + xs];
  }
  if constexpr (sizeof(T) == 4) {
    collide_f32(f, M.rho0_f, M.omega_f, fx, fy, M.alpha_f);
  } else {
    collide_f64(f, M.omega, fx, fy, M.alpha);
  }
#pragma unroll
  for (int l = 0; l < kQ; ++l) dst[(size_t)l * M.plane + (size_t)y * M.pitch + x] = f[l];
}

static dim3 grid2d(int nx, int ny, dim3 b) {
  return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y);
}

cudaError_t launch_step_scalar(int precision, const Member *d_members, int member, int nx,
                               int ny, int cur, cudaStream_t s) {
  dim3 b(64, 4);
  if (precision == 32)
    k_step_scalar<float><<<grid2d(nx, ny, b), b, 0, s>>>(d_members, member, cur);
  else
    k_step_scalar<double><<<grid2d(nx, ny, b), b, 0, s>>>(d_members, member, cur);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State conversion: init from (rho, u), public populations in and out,
// moment snapshots and the divergence flag.
// ---------------------------------------------------------------------------

// Storage of population l at cell x holds the value that streams to x + c_l:
// stored_l(x) = f_l(x + c_l, n).
template <typename T>
__global__ void k_init(const Member *__restrict__ members, int member, const double *rho,
                       const double *ux, const double *uy, int cur) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  T *dst = static_cast<T *>(M.pop[cur]);
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int xs = wrapi(x + cx_of(l), M.nx), ys = wrapi(y + cy_of(l), M.ny);
    const size_t c = (size_t)ys * M.nx + xs;
    const double r = rho[c], u = ux[c], v = uy[c];
    const double cu = cx_of(l) * u + cy_of(l) * v;
    const double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * (u * u + v * v);
    double val;
    if (sizeof(T) == 4)
      val = w_of(l) * ((r - M.rho0) + r * poly);  // deviation from t_l rho0
    else
      val = w_of(l) * r * (1.0 + poly);
    dst[(size_t)l * M.plane + (size_t)y * M.pitch + x] = (T)val;
  }
}

template <typename T>
__global__ void k_get_pop(const Member *__restrict__ members, int member, int cur, double *f) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(M.pop[cur]);
  const size_t N = (size_t)M.nx * M.ny;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int xs = wrapi(x - cx_of(l), M.nx), ys = wrapi(y - cy_of(l), M.ny);
    double v = (double)src[(size_t)l * M.plane + (size_t)ys * M.pitch + xs];
    if (sizeof(T) == 4) v += w_of(l) * M.rho0;
    f[(size_t)l * N + (size_t)y * M.nx + x] = v;
  }
}

template <typename T>
__global__ void k_set_pop(const Member *__restrict__ members, int member, int cur,
                          const double *f) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  T *dst = static_cast<T *>(M.pop[cur]);
  const size_t N = (size_t)M.nx * M.ny;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int xs = wrapi(x + cx_of(l), M.nx), ys = wrapi(y + cy_of(l), M.ny);
    double v = f[(size_t)l * N + (size_t)ys * M.nx + xs];
    if (sizeof(T) == 4) v -= w_of(l) * M.rho0;
    dst[(size_t)l * M.plane + (size_t)y * M.pitch + x] = (T)v;
  }
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

// (rho, j_x, j_y) of the pre-collision state, FP64, into d[3][ny*nx].
template <typename T>
__global__ void k_snapshot(const Member *__restrict__ members, int member, int cur, double *d) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(M.pop[cur]);
  T f[kQ];
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    int xs = x - cx_of(l), ys = y - cy_of(l);  // one-cell shifts: a single wrap
    xs = xs < 0 ? xs + M.nx : (xs >= M.nx ? xs - M.nx : xs);
    ys = ys < 0 ? ys + M.ny : (ys >= M.ny ? ys - M.ny : ys);
    f[l] = src[(size_t)l * M.plane + (size_t)ys * M.pitch + xs];
  }
  double r, jx, jy;
  if constexpr (sizeof(T) == 4) {
    // deviations: rho = rho0 + sum g (weights sum to 1), j = sum c g
    const int one[kQ] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    const float ax[6] = {f[1], f[5], f[8], f[3], f[6], f[7]};
    const float ay[6] = {f[2], f[5], f[6], f[4], f[7], f[8]};
    const int sgn[6] = {1, 1, 1, -1, -1, -1};
    r = M.rho0 + csum(f, one, kQ);
    jx = csum(ax, sgn, 6);
    jy = csum(ay, sgn, 6);
  } else {
    r = 0.0;
    jx = 0.0;
    jy = 0.0;
#pragma unroll
    for (int l = 0; l < kQ; ++l) {
      r += f[l];
      jx += cx_of(l) * f[l];
      jy += cy_of(l) * f[l];
    }
  }
  const size_t N = (size_t)M.nx * M.ny, c = (size_t)y * M.nx + x;
  d[c] = r;
  d[N + c] = jx;
  d[2 * N + c] = jy;
}

template <typename T>
__global__ void k_status(const Member *__restrict__ members, int member, int cur) {
  const Member &M = members[member];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= M.nx || y >= M.ny) return;
  const T *src = static_cast<const T *>(M.pop[cur]);
  double r = 0.0;
  bool bad = false;
#pragma unroll
  for (int l = 0; l < kQ; ++l) {
    const int xs = wrapi(x - cx_of(l), M.nx), ys = wrapi(y - cy_of(l), M.ny);
    const double v = (double)src[(size_t)l * M.plane + (size_t)ys * M.pitch + xs];
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

cudaError_t launch_init_fields(int precision, const Member *d_members, int member, int nx,
                               int ny, const double *rho, const double *ux,
                               const double *uy, int cur, cudaStream_t s) {
  LBM_DISPATCH(precision, k_init, d_members, member, rho, ux, uy, cur);
  return cudaGetLastError();
}

cudaError_t launch_get_populations(int precision, const Member *d_members, int member,
                                   int nx, int ny, int cur, double *f, cudaStream_t s) {
  LBM_DISPATCH(precision, k_get_pop, d_members, member, cur, f);
  return cudaGetLastError();
}

cudaError_t launch_set_populations(int precision, const Member *d_members, int member,
                                   int nx, int ny, int cur, const double *f, cudaStream_t s) {
  LBM_DISPATCH(precision, k_set_pop, d_members, member, cur, f);
  return cudaGetLastError();
}

cudaError_t launch_snapshot(int precision, const Member *d_members, int member, int nx,
                            int ny, int cur, double *dst, cudaStream_t s) {
  LBM_DISPATCH(precision, k_snapshot, d_members, member, cur, dst);
  return cudaGetLastError();
}

cudaError_t launch_status(int precision, const Member *d_members, int member, int nx,
                          int ny, int cur, cudaStream_t s) {
  LBM_DISPATCH(precision, k_status, d_members, member, cur);
  return cudaGetLastError();
}

}  // namespace lbm
