// gl_map.cu - multi-start MAP around the batched gradient (arXiv:2202.07663,
// Sec. 2.2-2.3): component-wise bijectors, the prior's log density and the
// Adam update, one warp per start, one lane per parameter, FP64.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/gigalens.h"
#include "gl_internal.h"
#include "gl_prior.cuh"

namespace {

using namespace gl::prior;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_map_inverse(int B, const float* __restrict__ theta, double* __restrict__ z, PriorTable P) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb)
    if (lane < GL_NPARAM) z[size_t(b) * GL_NPARAM + lane] = inv_bij(P.e[lane], double(theta[size_t(b) * GL_NPARAM + lane]));
}

__global__ void k_map_transform(int B, const double* __restrict__ z, float* __restrict__ theta, PriorTable P) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb)
    if (lane < GL_NPARAM) {
      double th, d, lj, dlj;
      bij(P.e[lane], z[size_t(b) * GL_NPARAM + lane], th, d, lj, dlj);
      theta[size_t(b) * GL_NPARAM + lane] = float(th);
    }
}

// Objective f(z) = -(log L + log p(g(z)) + log|J|) at the current z (Eq.
// obj-fun), its gradient, the Adam update (when m != null) and g(z_new).
__global__ void k_map_step(int B, double* __restrict__ z, double* __restrict__ m, double* __restrict__ v, double c1,
                           double c2, double lr, double b1, double b2, double eps, const double* __restrict__ loglik,
                           const double* __restrict__ grad, double* __restrict__ f_out, float* __restrict__ theta,
                           PriorTable P) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb) {
    const size_t i = size_t(b) * GL_NPARAM + lane;
    double part = 0.0, g = 0.0, zj = 0.0;
    if (lane < GL_NPARAM) {
      zj = z[i];
      double th, d, lj, dlj, lp, dlp;
      bij(P.e[lane], zj, th, d, lj, dlj);
      logpdf(P.e[lane], th, lp, dlp);
      part = lp + lj;
      g = -((grad[i] + dlp) * d + dlj);
    }
    const double tot = warp_sum(part);
    if (lane == 0 && f_out) f_out[b] = -(loglik[b] + tot);
    if (lane < GL_NPARAM) {
      if (m) {
        const double mi = b1 * m[i] + (1.0 - b1) * g;
        const double vi = b2 * v[i] + (1.0 - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        zj -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
        z[i] = zj;
      }
      if (theta) {
        double th, d, lj, dlj;
        bij(P.e[lane], zj, th, d, lj, dlj);
        theta[i] = float(th);
      }
    }
  }
}

// log p~(z) = log L + log p(g(z)) + log|J| (Eq. reparam-post) and its gradient in z.
__global__ void k_posterior(int B, const double* __restrict__ z, const double* __restrict__ loglik,
                            const double* __restrict__ grad, double* __restrict__ logp_out,
                            double* __restrict__ grad_z, PriorTable P) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb) {
    const size_t i = size_t(b) * GL_NPARAM + lane;
    double part = 0.0;
    if (lane < GL_NPARAM) {
      double th, d, lj, dlj, lp, dlp;
      bij(P.e[lane], z[i], th, d, lj, dlj);
      logpdf(P.e[lane], th, lp, dlp);
      part = lp + lj;
      if (grad) grad_z[i] = (grad[i] + dlp) * d + dlj;
    }
    const double tot = warp_sum(part);
    if (lane == 0) logp_out[b] = loglik[b] + tot;
  }
}

// The whitened posterior of the HMC preconditioning (Sec. 2.5), z = mu + L x
// with L lower triangular: one warp per chain, lane i for parameter i.
// k_whitened_transform forms z (the sums of gl_hmc_affine) and theta = g(z);
// k_whitened_posterior forms log p~(z) and its gradient in z (as k_posterior)
// and pulls the gradient back to x, grad_x = L^T grad_z (the sums of
// gl_hmc_affine_pullback). Two launches per evaluation instead of four.
constexpr int kWhitenedThreads = 32;

// The 22 x 22 factor into shared memory (blocks of kWhitenedThreads threads):
// each thread issues all of its loads before its first store, so the block
// waits for one round trip to L2 instead of one per row of the loop.
__device__ __forceinline__ void load_factor(double* sL, const double* __restrict__ Lc) {
  constexpr int N = GL_NPARAM * GL_NPARAM, PER = (N + kWhitenedThreads - 1) / kWhitenedThreads;
  double v[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = int(threadIdx.x) + u * kWhitenedThreads;
    v[u] = i < N ? Lc[i] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = int(threadIdx.x) + u * kWhitenedThreads;
    if (i < N) sL[i] = v[u];
  }
}

__global__ void __launch_bounds__(kWhitenedThreads) k_whitened_transform(int B, const double* __restrict__ x,
                                                                         const double* __restrict__ mu,
                                                                         const double* __restrict__ Lc,
                                                                         double* __restrict__ z,
                                                                         float* __restrict__ theta, PriorTable P) {
  constexpr int D = GL_NPARAM;
  __shared__ double sL[D * D];
  load_factor(sL, Lc);
  __syncthreads();
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb) {
    if (lane >= D) continue;
    const double* xb = x + size_t(b) * D;
    double acc = mu[lane];
    for (int j = 0; j <= lane; ++j) acc += sL[lane * D + j] * xb[j];
    z[size_t(b) * D + lane] = acc;
    double th, d, lj, dlj;
    bij(P.e[lane], acc, th, d, lj, dlj);
    theta[size_t(b) * D + lane] = float(th);
  }
}

// The leapfrog update of HMC on the whitened coordinates followed by
// k_whitened_transform at the new point: p += kick eps grad, x += eps M^-1 p
// (the arithmetic of gl_hmc_leapfrog), z = mu + L x, theta = g(z).
__global__ void __launch_bounds__(kWhitenedThreads) k_leapfrog_whitened(int B, double* __restrict__ x,
                                                                        double* __restrict__ p,
                                                                        const double* __restrict__ grad,
                                                                        const double* __restrict__ inv_mass,
                                                                        double eps_arg,
                                                                        const double* __restrict__ eps_dev,
                                                                        double kick, const double* __restrict__ mu,
                                                                        const double* __restrict__ Lc,
                                                                        double* __restrict__ z,
                                                                        float* __restrict__ theta, PriorTable P) {
  constexpr int D = GL_NPARAM;
  __shared__ double sL[D * D];
  load_factor(sL, Lc);
  __syncthreads();
  const double eps = eps_dev ? *eps_dev : eps_arg;
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < B; b += gridDim.x * wpb) {
    const size_t i = size_t(b) * D + lane;
    double xi = 0.0;
    if (lane < D) {
      const double pi = p[i] + kick * eps * grad[i];
      xi = x[i] + eps * inv_mass[lane] * pi;
      p[i] = pi;
      x[i] = xi;
    }
    double acc = lane < D ? mu[lane] : 0.0;
    for (int j = 0; j < D; ++j) {   // every lane shuffles; lanes >= D read no matrix row
      const double xj = __shfl_sync(0xffffffffu, xi, j);
      if (lane < D && j <= lane) acc += sL[lane * D + j] * xj;
    }
    if (lane < D) {
      z[i] = acc;
      double th, d, lj, dlj;
      bij(P.e[lane], acc, th, d, lj, dlj);
      theta[i] = float(th);
    }
  }
}

__global__ void __launch_bounds__(kWhitenedThreads) k_whitened_posterior(int B, const double* __restrict__ z,
                                                                         const double* __restrict__ loglik,
                                                                         const double* __restrict__ grad,
                                                                         const double* __restrict__ Lc,
                                                                         double* __restrict__ logp_out,
                                                                         double* __restrict__ grad_x, PriorTable P) {
  constexpr int D = GL_NPARAM;
  __shared__ double sL[D * D];
  __shared__ double sg[kWhitenedThreads / 32][32];
  load_factor(sL, Lc);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + w; b < B; b += gridDim.x * wpb) {
    const size_t i = size_t(b) * D + lane;
    double part = 0.0;
    if (lane < D) {
      double th, d, lj, dlj, lp, dlp;
      bij(P.e[lane], z[i], th, d, lj, dlj);
      logpdf(P.e[lane], th, lp, dlp);
      part = lp + lj;
      if (grad) sg[w][lane] = (grad[i] + dlp) * d + dlj;
    }
    const double tot = warp_sum(part);
    if (lane == 0) logp_out[b] = loglik[b] + tot;
    __syncwarp();
    if (grad && lane < D) {
      double acc = 0.0;
      for (int r = lane; r < D; ++r) acc += sL[r * D + lane] * sg[w][r];
      grad_x[i] = acc;
    }
    __syncwarp();
  }
}

// A leapfrog step after the first of a trajectory, in one launch: the
// gradient at the current point z (the sums of k_whitened_posterior, without
// log p~, which the trajectory does not need until its last point), then
// k_whitened_posterior's gradient into k_leapfrog_whitened's update and
// transform. z holds the current point on entry and the new one on exit: lane
// i reads and writes element i of its chain only, the read first.
__global__ void __launch_bounds__(kWhitenedThreads) k_leapfrog_whitened_chain(int B, double* __restrict__ x,
                                                                              double* __restrict__ p,
                                                                              double* __restrict__ z,
                                                                              const double* __restrict__ grad_theta,
                                                                              const double* __restrict__ inv_mass,
                                                                              double eps_arg,
                                                                              const double* __restrict__ eps_dev,
                                                                              double kick,
                                                                              const double* __restrict__ mu,
                                                                              const double* __restrict__ Lc,
                                                                              float* __restrict__ theta,
                                                                              PriorTable P) {
  constexpr int D = GL_NPARAM;
  __shared__ double sL[D * D];
  __shared__ double sg[kWhitenedThreads / 32][32];
  load_factor(sL, Lc);
  __syncthreads();
  const double eps = eps_dev ? *eps_dev : eps_arg;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int b = blockIdx.x * wpb + w; b < B; b += gridDim.x * wpb) {
    const size_t i = size_t(b) * D + lane;
    // this lane's state, loaded up front (lane i reads and writes element i only)
    double p0 = 0.0, x0 = 0.0, im = 0.0, m0 = 0.0;
    if (lane < D) {
      p0 = p[i];
      x0 = x[i];
      im = inv_mass[lane];
      m0 = mu[lane];
      double th, d, lj, dlj, lp, dlp;
      bij(P.e[lane], z[i], th, d, lj, dlj);
      logpdf(P.e[lane], th, lp, dlp);
      sg[w][lane] = (grad_theta[i] + dlp) * d + dlj;
    }
    __syncwarp();
    double xi = 0.0;
    if (lane < D) {
      double acc = 0.0;
      for (int r = lane; r < D; ++r) acc += sL[r * D + lane] * sg[w][r];
      const double g = acc;
      const double pi = p0 + kick * eps * g;
      xi = x0 + eps * im * pi;
      p[i] = pi;
      x[i] = xi;
    }
    double acc = lane < D ? m0 : 0.0;
    for (int j = 0; j < D; ++j) {   // every lane shuffles; lanes >= D read no matrix row
      const double xj = __shfl_sync(0xffffffffu, xi, j);
      if (lane < D && j <= lane) acc += sL[lane * D + j] * xj;
    }
    if (lane < D) {
      z[i] = acc;
      double th, d, lj, dlj;
      bij(P.e[lane], acc, th, d, lj, dlj);
      theta[i] = float(th);
    }
    __syncwarp();   // sg is rewritten for the warp's next chain
  }
}

// One warp (one start or chain) per block: the per-parameter arithmetic is
// FP64 (bijectors, prior densities), and GB300's FP64 pipe is narrow, so the
// chains are spread over as many SMs as there are (50 chains: 32 -> 9 us for
// the whitened posterior gradient against four warps per block).
constexpr int kMapThreads = 32;

int grid_for(int B) {
  return B < 1 ? 1 : (B > 8192 ? 8192 : B);
}

int finish(cudaStream_t st, const char* what) {
  cudaError_t e = gl_internal::hooks()->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, what);
}

}  // namespace

extern "C" {

int gl_map_inverse(int B, const float* theta, const gl_prior_entry* prior, double* z_out, void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!theta || !z_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_map_inverse<<<grid_for(B), kMapThreads, 0, st>>>(B, theta, z_out, P);
  return finish(st, "k_map_inverse");
}

int gl_map_transform(int B, const double* z, const gl_prior_entry* prior, float* theta_out, void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!z || !theta_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_map_transform<<<grid_for(B), kMapThreads, 0, st>>>(B, z, theta_out, P);
  return finish(st, "k_map_transform");
}

int gl_map_adam_step(int B, double* z, double* m, double* v, int t, double lr, double beta1, double beta2, double eps,
                     const double* loglik, const double* grad_theta, const gl_prior_entry* prior,
                     double* objective_out, float* theta_out, void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!z || !loglik || !grad_theta) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if ((m == nullptr) != (v == nullptr)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "m and v go together");
  if (m && t < 1) return gl_internal::set_error(GL_ERR_INVALID_ARG, "Adam step count t starts at 1");
  const double c1 = m ? 1.0 - pow(beta1, t) : 1.0, c2 = m ? 1.0 - pow(beta2, t) : 1.0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_map_step<<<grid_for(B), kMapThreads, 0, st>>>(B, z, m, v, c1, c2, lr, beta1, beta2, eps, loglik, grad_theta,
                                          objective_out, theta_out, P);
  return finish(st, "k_map_step");
}

int gl_posterior_grad(int B, const double* z, const double* loglik, const double* grad_theta,
                      const gl_prior_entry* prior, double* logp_out, double* grad_z_out, void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!z || !loglik || !logp_out || (grad_theta && !grad_z_out))
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_posterior<<<grid_for(B), kMapThreads, 0, st>>>(B, z, loglik, grad_theta, logp_out, grad_z_out, P);
  return finish(st, "k_posterior");
}

int gl_posterior_whitened_transform(int B, const double* x, const double* mu, const double* L,
                                    const gl_prior_entry* prior, double* z_out, float* theta_out, void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!x || !mu || !L || !z_out || !theta_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (z_out == x) return gl_internal::set_error(GL_ERR_INVALID_ARG, "z_out and x alias");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_whitened_transform<<<grid_for(B), kWhitenedThreads, 0, st>>>(B, x, mu, L, z_out, theta_out, P);
  return finish(st, "k_whitened_transform");
}

int gl_posterior_whitened_grad(int B, const double* z, const double* loglik, const double* grad_theta,
                               const double* L, const gl_prior_entry* prior, double* logp_out, double* grad_x_out,
                               void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!z || !loglik || !L || !logp_out || (grad_theta && !grad_x_out))
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (grad_theta && grad_x_out == grad_theta)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "grad_x_out and grad_theta alias");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_whitened_posterior<<<grid_for(B), kWhitenedThreads, 0, st>>>(B, z, loglik, grad_theta, L, logp_out, grad_x_out,
                                                                   P);
  return finish(st, "k_whitened_posterior");
}

int gl_hmc_leapfrog_whitened(int B, double* x, double* p, const double* grad, const double* inv_mass, double eps,
                             const double* eps_dev, double kick, const double* mu, const double* L,
                             const gl_prior_entry* prior, double* z_out, float* theta_out, void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!x || !p || !grad || !inv_mass || !mu || !L || !z_out || !theta_out)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (!eps_dev && !std::isfinite(eps)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "eps not finite");
  if (z_out == x) return gl_internal::set_error(GL_ERR_INVALID_ARG, "z_out and x alias");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_leapfrog_whitened<<<grid_for(B), kWhitenedThreads, 0, st>>>(B, x, p, grad, inv_mass, eps, eps_dev, kick, mu, L,
                                                                  z_out, theta_out, P);
  return finish(st, "k_leapfrog_whitened");
}

int gl_hmc_leapfrog_whitened_chain(int B, double* x, double* p, double* z, const double* grad_theta,
                                   const double* inv_mass, double eps, const double* eps_dev, double kick,
                                   const double* mu, const double* L, const gl_prior_entry* prior, float* theta_out,
                                   void* stream) {
  PriorTable P;
  int rc = load_table(prior, P);
  if (rc != GL_OK) return rc;
  if (B < 0) return gl_internal::set_error(GL_ERR_INVALID_ARG, "B < 0");
  if (B == 0) return GL_OK;
  if (!x || !p || !z || !grad_theta || !inv_mass || !mu || !L || !theta_out)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if (!eps_dev && !std::isfinite(eps)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "eps not finite");
  if (z == x || z == p || x == p || z == grad_theta || p == grad_theta || x == grad_theta)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "state arrays alias");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_leapfrog_whitened_chain<<<grid_for(B), kWhitenedThreads, 0, st>>>(B, x, p, z, grad_theta, inv_mass, eps, eps_dev,
                                                                        kick, mu, L, theta_out, P);
  return finish(st, "k_leapfrog_whitened_chain");
}

}  // extern "C"
