// Whole-grid balance quantities of one D2Q9 state without any device
// allocation: a variant of lbm_global_balance for callers that cannot obtain
// device memory from cudaMalloc (or from an allocator that calls it).  Its
// scratch lives in a file-scope __device__ array of fixed size, so the call
// needs neither a handle nor a workspace.
//
// Scratch use per call: the velocity field u = (j + F/2)/rho (2 doubles per
// cell), one partial-sum row per reduction block, and the 7 results.  Every
// call overwrites what it reads; nothing has to start at zero.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

namespace {

constexpr int kStaticBlocks = 512;
constexpr size_t kStaticDoubles =
    2 * (size_t)LBM_STATIC_MAX_CELLS + (size_t)kStaticBlocks * LBM_NGLOBAL + 8;

// Shared by every call on a device; it stays allocated until the process
// exits.  Host code must not use this symbol as a device address: it asks
// the runtime for the device address (cudaGetSymbolAddress) instead.
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};
thread_local char g_static_error[256] = "no error";

int fail_static(int code, const char *msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    snprintf(g_static_error, sizeof g_static_error, "%s: %s", msg, cudaGetErrorString(e));
  else
    snprintf(g_static_error, sizeof g_static_error, "%s", msg);
  return code;
}

struct SGrid {
  int nx, ny, kf, force;
  double nu, alpha, F0;
};

__device__ __forceinline__ int swrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// F_ext at (x, y): F0 (sin(2 pi kf y/ny), sin(2 pi kf x/nx)).
__device__ __forceinline__ void s_force(const SGrid &g, int x, int y, double &fx, double &fy) {
  if (g.force == 1) {
    fx = g.F0 * sinpi(2.0 * g.kf * (double)y / g.ny);
    fy = g.F0 * sinpi(2.0 * g.kf * (double)x / g.nx);
  } else {
    fx = 0.0;
    fy = 0.0;
  }
}

__device__ __forceinline__ void s_moments(const double *f, size_t N, size_t c, double &r,
                                          double &jx, double &jy) {
  r = 0.0;
  jx = 0.0;
  jy = 0.0;
#pragma unroll
  for (int l = 0; l < lbm::kQ; ++l) {
    const double v = f[(size_t)l * N + c];
    r += v;
    jx += lbm::cx_of(l) * v;
    jy += lbm::cy_of(l) * v;
  }
}

// Eq. (18) difference along x and y, periodic.
__device__ __forceinline__ double s_dx(const double *A, const SGrid &g, int x, int y) {
  const double *r = A + (size_t)y * g.nx;
  auto a = [&](int d) { return r[swrap(x + d, g.nx)]; };
  return 0.8 * (a(1) - a(-1)) - 0.2 * (a(2) - a(-2)) + (4.0 / 105.0) * (a(3) - a(-3)) -
         (1.0 / 280.0) * (a(4) - a(-4));
}
__device__ __forceinline__ double s_dy(const double *A, const SGrid &g, int x, int y) {
  auto a = [&](int d) { return A[(size_t)swrap(y + d, g.ny) * g.nx + x]; };
  return 0.8 * (a(1) - a(-1)) - 0.2 * (a(2) - a(-2)) + (4.0 / 105.0) * (a(3) - a(-3)) -
         (1.0 / 280.0) * (a(4) - a(-4));
}

__global__ void k_static_velocity(SGrid g, const double *f, double *scratch) {
  const size_t N = (size_t)g.nx * g.ny;
  double *U = scratch, *V = scratch + N;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    double r, jx, jy, fx, fy;
    s_moments(f, N, c, r, jx, jy);
    s_force(g, x, y, fx, fy);
    U[c] = (jx + 0.5 * (fx - g.alpha * jx)) / r;
    V[c] = (jy + 0.5 * (fy - g.alpha * jy)) / r;
  }
}

__global__ void k_static_reduce(SGrid g, const double *f, double *scratch) {
  const size_t N = (size_t)g.nx * g.ny;
  const double *U = scratch, *V = scratch + N;
  double *partials = scratch + 2 * (size_t)LBM_STATIC_MAX_CELLS;
  double acc[LBM_NGLOBAL] = {0, 0, 0, 0, 0, 0, 0};
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    double r, jx, jy, fx, fy;
    s_moments(f, N, c, r, jx, jy);
    s_force(g, x, y, fx, fy);
    const double Fx = fx - g.alpha * jx, Fy = fy - g.alpha * jy;
    const double u = U[c], v = V[c];
    const double dxu = s_dx(U, g, x, y), dyu = s_dy(U, g, x, y);
    const double dxv = s_dx(V, g, x, y), dyv = s_dy(V, g, x, y);
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
  __shared__ double sh[LBM_NGLOBAL][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < LBM_NGLOBAL; ++q) {
    double a = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[q][wid] = a;
  }
  __syncthreads();
  if (threadIdx.x < LBM_NGLOBAL) {
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a += sh[threadIdx.x][k];
    partials[(size_t)blockIdx.x * LBM_NGLOBAL + threadIdx.x] = a;
  }
}

__global__ void k_static_final(int nblocks, size_t N, double *scratch) {
  const double *partials = scratch + 2 * (size_t)LBM_STATIC_MAX_CELLS;
  double *out = scratch + 2 * (size_t)LBM_STATIC_MAX_CELLS + (size_t)kStaticBlocks * LBM_NGLOBAL;
  const int q = threadIdx.x;
  if (q >= LBM_NGLOBAL) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) a += partials[(size_t)b * LBM_NGLOBAL + q];
  out[q] = q < 3 ? a : a / (double)N;
}

// Device address of the scratch array on the current device, looked up once
// per device and kept for the life of the process (a device reset after the
// first call would leave it stale; the header says so).
int scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_static(LBM_ERR_CUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return fail_static(LBM_ERR_ARG, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return fail_static(LBM_ERR_CUDA, "cudaGetSymbolAddress", e);
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_global_balance_static(const double *f, int nx, int ny,
                                         const lbm_member_cfg *m, double *out,
                                         void *cuda_stream) {
  if (!f) return fail_static(LBM_ERR_ARG, "f is NULL");
  if (!m) return fail_static(LBM_ERR_ARG, "m is NULL");
  if (!out) return fail_static(LBM_ERR_ARG, "out is NULL");
  if (nx < 1 || ny < 1) return fail_static(LBM_ERR_ARG, "grid must be at least 1 x 1");
  if ((long long)nx * ny > (long long)LBM_STATIC_MAX_CELLS)
    return fail_static(LBM_ERR_ARG,
                       "grid larger than LBM_STATIC_MAX_CELLS cells: use lbm_global_balance");
  if (!(m->tau > 0.5) || !std::isfinite(m->tau) || (m->force_kind != 0 && m->force_kind != 1) ||
      m->collision != 0 || !std::isfinite(m->F0) || !std::isfinite(m->alpha))
    return fail_static(LBM_ERR_ARG, "invalid member parameters");
  double *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != LBM_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  SGrid g;
  g.nx = nx;
  g.ny = ny;
  g.kf = m->kf;
  g.force = m->force_kind;
  g.nu = (m->tau - 0.5) / 3.0;
  g.alpha = m->alpha;
  g.F0 = m->F0;
  const size_t N = (size_t)nx * ny;
  int nb = (int)((N + 255) / 256);
  if (nb > kStaticBlocks) nb = kStaticBlocks;
  k_static_velocity<<<nb, 256, 0, s>>>(g, f, scratch);
  k_static_reduce<<<nb, 256, 0, s>>>(g, f, scratch);
  k_static_final<<<1, 32, 0, s>>>(nb, N, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_static(LBM_ERR_CUDA, "kernel launch", e);
  const double *res = scratch + 2 * (size_t)LBM_STATIC_MAX_CELLS + (size_t)kStaticBlocks * LBM_NGLOBAL;
  e = cudaMemcpyAsync(out, res, sizeof(double) * LBM_NGLOBAL, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail_static(LBM_ERR_CUDA, "copy of the results", e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_static(LBM_ERR_CUDA, "stream synchronisation", e);
  return LBM_OK;
}

extern "C" const char *lbm_static_last_error(void) { return g_static_error; }
