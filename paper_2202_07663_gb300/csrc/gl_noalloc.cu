// gl_noalloc.cu - log-likelihood + gradient that allocates no memory.
//
// Some callers cannot call cudaMalloc at the time they evaluate the
// likelihood: code running inside a custom allocator or memory-pool callback
// (a call back into the allocator would re-enter it), processes whose device
// memory is fully pre-reserved by another framework's caching allocator, and
// hosts that forbid allocation after start-up (real-time or certified
// pipelines). gl_loglik_grad_noalloc serves them: it runs the same kernels as
// gl_loglik_grad, with the scratch those kernels need (per-vector constants,
// the per-vector image work buffer and the per-tile gradient partials) taken
// from one file-scope device array instead of memory the library allocates.
#include <cuda_runtime.h>

#include <cstdio>

#include "gl_device.cuh"
#include "gl_internal.h"
#include "gl_launch.h"

namespace {

// Size of the static scratch array. Every GPU that loads the library holds
// it until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Device address of the array on the current device. The host-side name of
// the array is not a device address, so it is looked up with the device
// current, on every call: the lookup allocates nothing, and no address is
// kept that a reset of the device's context could leave stale.
int scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return gl_internal::cuda_error(e, "cudaGetSymbolAddress(static scratch)");
  *out = p;
  return GL_OK;
}

}  // namespace

extern "C" {

int gl_loglik_grad_noalloc(gl_system* sys, const float* params, int B, double* loglik_out, double* chi2_out,
                           double* grad_out, void* stream) {
  if (!sys) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null gl_system");
  if (B < 0 || B > (1 << 24)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B outside [0, 2^24]");
  int rc = gl_internal::system_device_check(sys);
  if (rc != GL_OK) return rc;
  if (B == 0) return GL_OK;
  if (!params || !loglik_out || !grad_out)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null params, loglik_out or grad_out");
  gl::Seg g = gl_internal::seg_without_scratch(sys, params, B);
  const size_t vc_bytes = align256(sizeof(gl::VecConst) * size_t(B));
  const size_t work_bytes = align256(sizeof(float) * size_t(B) * g.H * g.W);
  const size_t part_bytes = align256(sizeof(double) * size_t(B) * g.ntiles * gl::NACC);
  const size_t need = vc_bytes + work_bytes + part_bytes;
  if (need > kNoAllocScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof(msg), "B = %d needs %zu bytes of static scratch; the limit is %zu bytes", B, need,
             kNoAllocScratchBytes);
    return gl_internal::set_error(GL_ERR_INVALID_ARG, msg);
  }
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc != GL_OK) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  // Every element of these buffers is written before it is read within one
  // call (setup writes all constants, the forward ray kernel every pixel,
  // the adjoint ray kernel every tile partial), so nothing needs clearing.
  g.vc = reinterpret_cast<gl::VecConst*>(p);
  g.work = reinterpret_cast<float*>(p + vc_bytes);
  g.partial = reinterpret_cast<double*>(p + vc_bytes + work_bytes);
  g.loglik = loglik_out;
  g.chi2 = chi2_out;
  g.grad = grad_out;
  cudaError_t e = gl::launch_one(g, gl::MODE_GRAD, static_cast<cudaStream_t>(stream), gl_internal::hooks());
  if (e != cudaSuccess) return gl_internal::cuda_error(e, "kernel launch");
  return GL_OK;
}

}  // extern "C"
