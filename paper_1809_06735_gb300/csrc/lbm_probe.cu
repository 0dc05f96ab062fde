// Arithmetic-throughput probe for the roofline of the ALU-bound kernels (no
// counterpart in the paper): independent chains of fused multiply-adds in
// FP64 or FP32 over every SM, timed with CUDA events on the caller's stream.
// The FP64 step and the adjoint on GB300 are bounded by its FP64 pipe, the
// entropic collision by the FP32 issue rate; this gives the measured
// ceiling they are reported against.
#include "lbm_internal.cuh"

namespace lbm {

namespace {

__device__ double g_probe_sink64;
__device__ float g_probe_sink32;

template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T seed, T *sink) {
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = seed + (T)(threadIdx.x & 7) + (T)k;
  const T m = (T)0.9999999, c = (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], m, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  if (s == (T)-1) *sink = s;  // never taken (every chain stays positive): keeps them live
}

template <typename T>
cudaError_t time_chains(int iters, T *sink, cudaStream_t s, double *flops_per_s) {
  int sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  constexpr int kChains = 8, kThreads = 256, kCtasPerSm = 8;
  const int grid = sms * kCtasPerSm;
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  k_fma_chains<T, kChains><<<grid, kThreads, 0, s>>>(iters / 8, (T)1, sink);  // warm-up
  cudaEventRecord(a, s);
  k_fma_chains<T, kChains><<<grid, kThreads, 0, s>>>(iters, (T)1, sink);
  cudaEventRecord(b, s);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  const double fmas = (double)grid * kThreads * kChains * (double)iters;
  *flops_per_s = 2.0 * fmas / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace

cudaError_t probe_fma_rate(int bits, cudaStream_t s, double *flops_per_s) {
  if (bits == 64) {
    double *sink = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&sink, g_probe_sink64);
    if (e != cudaSuccess) return e;
    return time_chains<double>(4096, sink, s, flops_per_s);
  }
  float *sink = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void **)&sink, g_probe_sink32);
  if (e != cudaSuccess) return e;
  return time_chains<float>(131072, sink, s, flops_per_s);
}

}  // namespace lbm
