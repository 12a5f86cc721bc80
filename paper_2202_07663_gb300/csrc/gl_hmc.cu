// gl_hmc.cu - leapfrog and Metropolis kernels of Hamiltonian Monte Carlo
// (arXiv:2202.07663, Sec. 2.5) around the batched log-likelihood gradient.
//
// Chain state (positions q, momenta p, log density, its gradient) is FP64 on
// the device; positions are handed to the likelihood as FP32. The Hamiltonian
// H = -log p(q) + 1/2 p^T M^-1 p and the accept test run in FP64 on the GPU.
// Random numbers (momenta, accept uniforms) are drawn by the caller.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/gigalens.h"
#include "gl_internal.h"

namespace {

// p += kick * eps * grad;  q += eps * M^-1 p;  q32 = float(q). One thread per component.
__global__ void k_hmc_leapfrog(int n, int d, double* __restrict__ q, double* __restrict__ p,
                               const double* __restrict__ grad, const double* __restrict__ inv_mass, double eps,
                               double kick, float* __restrict__ q32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double pi = p[i] + kick * eps * grad[i];
    const double qi = q[i] + eps * inv_mass[i % d] * pi;
    p[i] = pi;
    q[i] = qi;
    q32[i] = float(qi);
  }
}

// Final half kick, Hamiltonians of the start and end points, accept/reject.
// One warp per chain.
__global__ void k_hmc_finish(int B, int d, const double* __restrict__ p0, const double* __restrict__ logp0,
                             double* __restrict__ p, const double* __restrict__ grad_new,
                             const double* __restrict__ logp_new, const double* __restrict__ q_new,
                             const double* __restrict__ inv_mass, const double* __restrict__ log_u, double eps,
                             double* __restrict__ q, double* __restrict__ logp, double* __restrict__ grad,
                             int* __restrict__ accepted) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb) {
    double k0 = 0.0, k1 = 0.0;
    for (int j = lane; j < d; j += 32) {
      const size_t i = size_t(b) * d + j;
      const double pj = p[i] + 0.5 * eps * grad_new[i];
      p[i] = pj;
      k0 += p0[i] * p0[i] * inv_mass[j];
      k1 += pj * pj * inv_mass[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      k0 += __shfl_xor_sync(0xffffffffu, k0, o);
      k1 += __shfl_xor_sync(0xffffffffu, k1, o);
    }
    const double h0 = -logp0[b] + 0.5 * k0;
    const double h1 = -logp_new[b] + 0.5 * k1;
    const bool acc = isfinite(h1) && isfinite(h0) && (log_u[b] < h0 - h1);
    if (acc) {
      for (int j = lane; j < d; j += 32) {
        const size_t i = size_t(b) * d + j;
        q[i] = q_new[i];
        grad[i] = grad_new[i];
      }
    }
    if (lane == 0) {
      if (acc) logp[b] = logp_new[b];
      accepted[b] = acc ? 1 : 0;
    }
  }
}

int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return int(g < 4096 ? (g < 1 ? 1 : g) : 4096);
}

}  // namespace

extern "C" {

int gl_hmc_leapfrog(int B, int d, double* q, double* p, const double* grad, const double* inv_mass, double eps,
                    double kick, float* q32_out, void* stream) {
  if (B < 0 || d < 1 || d > 4096) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad B or d");
  if (B == 0) return GL_OK;
  if (!q || !p || !grad || !inv_mass || !q32_out)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (!std::isfinite(eps) || !std::isfinite(kick)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "eps or kick");
  const long long n = (long long)B * d;
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_hmc_leapfrog<<<grid_for(n, 256), 256, 0, st>>>(int(n), d, q, p, grad, inv_mass, eps, kick, q32_out);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_hmc_leapfrog");
}

int gl_hmc_finish(int B, int d, const double* p0, const double* logp0, double* p, const double* grad_new,
                  const double* logp_new, const double* q_new, const double* inv_mass, const double* log_u, double eps,
                  double* q, double* logp, double* grad, int* accepted, void* stream) {
  if (B < 0 || d < 1 || d > 4096) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad B or d");
  if (B == 0) return GL_OK;
  if (!p0 || !logp0 || !p || !grad_new || !logp_new || !q_new || !inv_mass || !log_u || !q || !logp || !grad ||
      !accepted)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_hmc_finish<<<grid_for((long long)B * 32, 128), 128, 0, st>>>(B, d, p0, logp0, p, grad_new, logp_new, q_new,
                                                                  inv_mass, log_u, eps, q, logp, grad, accepted);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_hmc_finish");
}

}  // extern "C"
