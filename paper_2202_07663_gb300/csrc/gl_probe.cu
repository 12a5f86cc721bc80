// gl_probe.cu - measured throughput of the two pipes the likelihood kernels
// are bound by: packed FP32 fused multiply-add and the special-function
// unit's ex2. The benchmark divides its kernels' algorithmic work by these
// rates (taken at the clock the GPU runs at), so the roofline's denominator
// is a measurement on the same device rather than a nominal figure.
#include <cuda_runtime.h>

#include "../../include/gigalens.h"
#include "gl_device.cuh"
#include "gl_internal.h"

namespace {

constexpr int kChains = 16;         // independent dependency chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

// kChains chains of packed FMAs, a <- a m + c (|m| < 1 keeps them finite).
__global__ void __launch_bounds__(kThreads) k_peak_ffma2(int iters, float* out) {
  float2 a[kChains];
  const float2 m = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = make_float2(threadIdx.x * 1e-3f + j, 0.5f * j);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j].x + a[j].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// kChains chains of a <- 2^(-a), which stays in (1/2, 1).
__global__ void __launch_bounds__(kThreads) k_peak_ex2(int iters, float* out) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 0.1f * (j + 1) + threadIdx.x * 1e-6f;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = gl::ex2(-a[j]);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int gl_profile_peak(int kind, double* rate_out) {
  if (!rate_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null rate_out");
  if (kind != GL_PEAK_FP32_FMA && kind != GL_PEAK_MUFU_EX2)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "unknown peak kind");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return gl_internal::cuda_error(e, "device query");
  const int grid = sms * kBlocksPerSM;
  const int iters = kind == GL_PEAK_FP32_FMA ? 4096 : 1024;   // a multiple of the unroll
  float* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaMalloc(&out, sizeof(float) * size_t(grid) * kThreads)) != cudaSuccess)
    return gl_internal::cuda_error(e, "probe buffer");
  float best = 0.f;
  if ((e = cudaEventCreate(&a)) == cudaSuccess && (e = cudaEventCreate(&b)) == cudaSuccess) {
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {   // the first launch warms up, the best of the rest counts
      cudaEventRecord(a, 0);
      if (kind == GL_PEAK_FP32_FMA) k_peak_ffma2<<<grid, kThreads>>>(iters, out);
      else k_peak_ex2<<<grid, kThreads>>>(iters, out);
      gl_internal::count_launches(1);
      cudaEventRecord(b, 0);
      e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return gl_internal::cuda_error(e, "peak probe");
  const double per_thread = kind == GL_PEAK_FP32_FMA ? double(iters) * kChains * 2 * 2   // 2 lanes, FMA = 2 flops
                                                     : double(iters) * kChains;
  *rate_out = per_thread * grid * kThreads / (double(best) * 1e-3);
  return GL_OK;
}
