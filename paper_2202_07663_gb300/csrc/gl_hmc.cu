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
// eps from *eps_dev when given (a value a replayed graph reads at run time).
__global__ void k_hmc_leapfrog(long long n, int d, double* __restrict__ q, double* __restrict__ p,
                               const double* __restrict__ grad, const double* __restrict__ inv_mass, double eps_arg,
                               const double* __restrict__ eps_dev, double kick, float* __restrict__ q32) {
  const double eps = eps_dev ? *eps_dev : eps_arg;
  // 64-bit index: B * d may exceed the int range
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double pi = p[i] + kick * eps * grad[i];
    const double qi = q[i] + eps * inv_mass[i % d] * pi;
    p[i] = pi;
    q[i] = qi;
    if (q32) q32[i] = float(qi);
  }
}

// Final half kick, Hamiltonians of the start and end points, accept/reject.
// One warp per chain.
__global__ void k_hmc_finish(int B, int d, const double* __restrict__ p0, const double* __restrict__ logp0,
                             double* __restrict__ p, const double* __restrict__ grad_new,
                             const double* __restrict__ logp_new, const double* __restrict__ q_new,
                             const double* __restrict__ inv_mass, const double* __restrict__ log_u, double eps,
                             double* __restrict__ q, double* __restrict__ logp, double* __restrict__ grad,
                             int* __restrict__ accepted, double* __restrict__ accept_prob) {
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
      if (accept_prob) accept_prob[b] = (isfinite(h1) && isfinite(h0)) ? fmin(1.0, exp(h0 - h1)) : 0.0;
    }
  }
}

// Whitened coordinates for a dense preconditioner: z = mu + L x with L lower
// triangular (row-major d x d), and the gradient pull-back g_x = L^T g_z.
// One warp per chain; L staged in shared memory.
__global__ void k_affine(int B, int d, const double* __restrict__ x, const double* __restrict__ mu,
                         const double* __restrict__ Lc, double* __restrict__ z, float* __restrict__ z32) {
  extern __shared__ double sL[];
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) sL[i] = Lc[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb) {
    const double* xb = x + size_t(b) * d;
    for (int i = lane; i < d; i += 32) {
      double acc = mu[i];
      for (int j = 0; j <= i; ++j) acc += sL[i * d + j] * xb[j];
      z[size_t(b) * d + i] = acc;
      if (z32) z32[size_t(b) * d + i] = float(acc);
    }
  }
}

__global__ void k_affine_pullback(int B, int d, const double* __restrict__ gz, const double* __restrict__ Lc,
                                  double* __restrict__ gx) {
  extern __shared__ double sL[];
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) sL[i] = Lc[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb) {
    const double* gb = gz + size_t(b) * d;
    for (int j = lane; j < d; j += 32) {
      double acc = 0.0;
      for (int i = j; i < d; ++i) acc += sL[i * d + j] * gb[i];
      gx[size_t(b) * d + j] = acc;
    }
  }
}

// ChEES gradient of Hoffman, Radul & Sountsov (2021) for the trajectory-length
// adaptation: per chain a = |q' - m'|^2 - |q - m|^2 and c = (q' - m') . M^-1 p',
// out = [sum w t a c / sum w, sum w a^2/4 / sum w, sum w], w the acceptance
// probability; a chain with a non-finite proposal, end momentum or weight
// has no weight and is left out of the proposals' mean m'. One block; fixed
// thread-to-chain mapping and a fixed reduction tree (reproducible).
constexpr int kCheesThreads = 256;

__global__ void __launch_bounds__(kCheesThreads) k_hmc_chees(int B, int d, const double* __restrict__ q_prev,
                                                             const double* __restrict__ q_prop,
                                                             const double* __restrict__ p_prop,
                                                             const double* __restrict__ inv_mass,
                                                             const double* __restrict__ w, double t,
                                                             double* __restrict__ out) {
  __shared__ unsigned char ok[GL_HMC_CHEES_MAX_B];
  __shared__ double m[GL_HMC_CHEES_MAX_D], mp[GL_HMC_CHEES_MAX_D];
  __shared__ double red[3][kCheesThreads];
  __shared__ int s_nok;
  const int tid = threadIdx.x;
  if (tid == 0) s_nok = 0;
  __syncthreads();
  int my_ok = 0;
  for (int b = tid; b < B; b += blockDim.x) {
    bool f = isfinite(w[b]);
    for (int j = 0; j < d && f; ++j) {
      const size_t i = size_t(b) * d + j;
      f = isfinite(q_prop[i]) && isfinite(p_prop[i]);
    }
    ok[b] = f ? 1 : 0;
    my_ok += f ? 1 : 0;
  }
  atomicAdd(&s_nok, my_ok);   // integer count: order does not matter
  __syncthreads();
  const int nok = s_nok;
  for (int j = tid; j < d; j += blockDim.x) {
    double a = 0.0, ap = 0.0;
    for (int b = 0; b < B; ++b) {
      a += q_prev[size_t(b) * d + j];
      if (ok[b]) ap += q_prop[size_t(b) * d + j];
    }
    m[j] = a / double(B);
    mp[j] = nok > 0 ? ap / double(nok) : 0.0;
  }
  __syncthreads();
  double sg = 0.0, sc = 0.0, sw = 0.0;
  for (int b = tid; b < B; b += blockDim.x) {
    if (!ok[b]) continue;
    double x2 = 0.0, y2 = 0.0, c = 0.0;
    for (int j = 0; j < d; ++j) {
      const size_t i = size_t(b) * d + j;
      const double dx = q_prop[i] - mp[j], dy = q_prev[i] - m[j];
      x2 += dx * dx;
      y2 += dy * dy;
      c += dx * inv_mass[j] * p_prop[i];
    }
    const double a = x2 - y2, wb = w[b];
    sg += wb * t * a * c;
    sc += wb * 0.25 * a * a;
    sw += wb;
  }
  red[0][tid] = sg;
  red[1][tid] = sc;
  red[2][tid] = sw;
  __syncthreads();
  for (int o = kCheesThreads / 2; o > 0; o >>= 1) {
    if (tid < o) {
      red[0][tid] += red[0][tid + o];
      red[1][tid] += red[1][tid + o];
      red[2][tid] += red[2][tid + o];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double W = red[2][0];
    out[0] = W > 0.0 ? red[0][0] / W : 0.0;
    out[1] = W > 0.0 ? red[1][0] / W : 0.0;
    out[2] = W;
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
  if (!q || !p || !grad || !inv_mass) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (!std::isfinite(eps) || !std::isfinite(kick)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "eps or kick");
  const long long n = (long long)B * d;
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_hmc_leapfrog<<<grid_for(n, 256), 256, 0, st>>>(n, d, q, p, grad, inv_mass, eps, nullptr, kick, q32_out);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_hmc_leapfrog");
}

int gl_hmc_leapfrog_dev(int B, int d, double* q, double* p, const double* grad, const double* inv_mass,
                        const double* eps_dev, double kick, float* q32_out, void* stream) {
  if (B < 0 || d < 1 || d > 4096) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad B or d");
  if (B == 0) return GL_OK;
  if (!q || !p || !grad || !inv_mass || !eps_dev) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (!std::isfinite(kick)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "kick");
  const long long n = (long long)B * d;
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_hmc_leapfrog<<<grid_for(n, 256), 256, 0, st>>>(n, d, q, p, grad, inv_mass, 0.0, eps_dev, kick, q32_out);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_hmc_leapfrog");
}

int gl_hmc_finish(int B, int d, const double* p0, const double* logp0, double* p, const double* grad_new,
                  const double* logp_new, const double* q_new, const double* inv_mass, const double* log_u, double eps,
                  double* q, double* logp, double* grad, int* accepted, double* accept_prob, void* stream) {
  if (B < 0 || d < 1 || d > 4096) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad B or d");
  if (B == 0) return GL_OK;
  if (!p0 || !logp0 || !p || !grad_new || !logp_new || !q_new || !inv_mass || !log_u || !q || !logp || !grad ||
      !accepted)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_hmc_finish<<<grid_for((long long)B * 32, 128), 128, 0, st>>>(B, d, p0, logp0, p, grad_new, logp_new, q_new,
                                                                  inv_mass, log_u, eps, q, logp, grad, accepted,
                                                                  accept_prob);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_hmc_finish");
}

int gl_hmc_chees(int B, int d, const double* q_prev, const double* q_prop, const double* p_prop,
                 const double* inv_mass, const double* accept_prob, double t, double* out, void* stream) {
  if (B < 1 || B > GL_HMC_CHEES_MAX_B || d < 1 || d > GL_HMC_CHEES_MAX_D)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad B or d");
  if (!q_prev || !q_prop || !p_prop || !inv_mass || !accept_prob || !out)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (!std::isfinite(t)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "t not finite");
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_hmc_chees<<<1, kCheesThreads, 0, st>>>(B, d, q_prev, q_prop, p_prop, inv_mass, accept_prob, t, out);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_hmc_chees");
}

int gl_hmc_affine(int B, int d, const double* x, const double* mu, const double* L, double* z_out, float* z32_out,
                  void* stream) {
  if (B < 0 || d < 1 || d > GL_HMC_AFFINE_MAX_D) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad B or d");
  if (B == 0) return GL_OK;
  if (!x || !mu || !L || !z_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (x == z_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "x and z_out alias");
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_affine<<<grid_for((long long)B * 32, 128), 128, size_t(d) * d * sizeof(double), st>>>(B, d, x, mu, L, z_out,
                                                                                           z32_out);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_affine");
}

int gl_hmc_affine_pullback(int B, int d, const double* grad_z, const double* L, double* grad_x_out, void* stream) {
  if (B < 0 || d < 1 || d > GL_HMC_AFFINE_MAX_D) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad B or d");
  if (B == 0) return GL_OK;
  if (!grad_z || !L || !grad_x_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (grad_z == grad_x_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "grad_z and grad_x_out alias");
  gl::Hooks* h = gl_internal::hooks();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->before(GL_K_OTHER, st);
  k_affine_pullback<<<grid_for((long long)B * 32, 128), 128, size_t(d) * d * sizeof(double), st>>>(B, d, grad_z, L,
                                                                                                    grad_x_out);
  cudaError_t e = h->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, "k_affine_pullback");
}

}  // extern "C"
