// gl_vi.cu - full-rank variational inference around the batched gradient
// (arXiv:2202.07663, Sec. 2.4): q = N(mu, L L^T) over the unconstrained
// parameters, L from the Cholesky bijector (lower triangle, exponentiated
// diagonal), the ELBO loss E_q[log q - log p~] and its gradient by the
// score-function estimator of Eq. elbo-grad or the reparameterised one.
//
// phi = [mu (d), u (d(d+1)/2)], u packed row by row: u[i(i+1)/2 + j] is
// L[i][j] for j < i and log L[i][i] for j = i.
//
// Both estimators reduce to sample moments of the draws eps_s:
//   score:    f_s = log q(z_s) - log p~(z_s), log q(z_s) = -|eps_s|^2/2 - sum u_ii - d/2 log 2 pi
//             d/dmu = L^-T mean(f eps);  d/dL = lower(L^-T mean(f eps eps^T)) - mean(f) diag(1/L_ii)
//   pathwise: d/dmu = -mean(grad_z);     d/dL_ij = -mean(grad_z_i eps_j) - delta_ij / L_ii
// and d/du_ii = L_ii d/dL_ii. k_vi_moments sums the moments per block over
// fixed chunks of 32 draws into the caller's workspace (no atomics: the sums
// are reproducible run to run); k_vi_finish adds the blocks' sums in order,
// forms the gradient, and applies Adam. FP64 throughout (a few hundred
// thousand FMAs per iteration, next to the likelihood's ~1e9).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/gigalens.h"
#include "gl_internal.h"
#include "gl_prior.cuh"

namespace {

using namespace gl::prior;

constexpr int kChunk = 32;                 // draws staged per pass
constexpr int kThreads = 256;
constexpr int kMaxQ = 1 + GL_VI_MAX_D + GL_VI_MAX_D * (GL_VI_MAX_D + 1) / 2;
constexpr int kSlots = (kMaxQ + kThreads - 1) / kThreads;
constexpr int kMaxBlocks = 152;
constexpr double kLn2Pi = 1.83787706640934548356;

__host__ __device__ inline int tri(int i) { return i * (i + 1) / 2; }

int n_blocks(int n) {
  const int c = (n + kChunk - 1) / kChunk;
  return c < 1 ? 1 : (c > kMaxBlocks ? kMaxBlocks : c);
}

// z = mu + L eps per draw; theta = g(z) (float) when a prior is given,
// (float) z when not. One warp per draw, lanes over components.
__global__ void k_vi_sample(int n, int d, const double* __restrict__ eps, const double* __restrict__ phi,
                            double* __restrict__ z, float* __restrict__ theta, PriorTable P, int use_prior) {
  __shared__ double sphi[GL_VI_MAX_D + GL_VI_MAX_D * (GL_VI_MAX_D + 1) / 2];
  const int np = d + tri(d);
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    double x = phi[i];
    if (i >= d) {
      const int k = i - d;  // position in the packed triangle; diagonal where k == tri(row) + row
      int r = int((sqrt(8.0 * k + 1.0) - 1.0) * 0.5);
      while (tri(r + 1) <= k) ++r;
      while (tri(r) > k) --r;
      if (k - tri(r) == r) x = exp(x);
    }
    sphi[i] = x;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int s = blockIdx.x * wpb + (threadIdx.x >> 5); s < n; s += gridDim.x * wpb) {
    const double* e = eps + size_t(s) * d;
    for (int i = lane; i < d; i += 32) {
      double acc = sphi[i];
      const double* Li = sphi + d + tri(i);
      for (int j = 0; j <= i; ++j) acc += Li[j] * e[j];
      z[size_t(s) * d + i] = acc;
      if (theta) {
        if (use_prior) {
          double th, dth, lj, dlj;
          bij(P.e[i], acc, th, dth, lj, dlj);
          theta[size_t(s) * d + i] = float(th);
        } else {
          theta[size_t(s) * d + i] = float(acc);
        }
      }
    }
  }
}

// Per-block sums of the estimator's moments over the block's chunks of draws.
// Accumulator q: 0 -> sum c0_s; 1..d -> sum c1_sj; then the packed lower
// triangle (i, j <= i) -> sum c2_si eps_sj, where
//   score:    c0 = f_s, c1_sj = f_s eps_sj, c2_si = f_s eps_si
//   pathwise: c0 = f_s, c1_sj = grad_z_sj,  c2_si = grad_z_si
__global__ void __launch_bounds__(kThreads) k_vi_moments(int n, int d, const double* __restrict__ eps,
                                                         const double* __restrict__ logp,
                                                         const double* __restrict__ grad_z,
                                                         const double* __restrict__ phi, int pathwise,
                                                         double* __restrict__ partial) {
  __shared__ double se[kChunk][GL_VI_MAX_D];
  __shared__ double sc[kChunk][GL_VI_MAX_D];
  __shared__ double sf[kChunk];
  __shared__ double s_logdet;
  const int Q = 1 + d + tri(d);
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < d; ++i) a += phi[d + tri(i) + i];
    s_logdet = a;  // sum log L_ii
  }
  // this thread's accumulators and their (kind, i, j)
  double acc[kSlots];
  int qi[kSlots], qj[kSlots];
#pragma unroll
  for (int k = 0; k < kSlots; ++k) {
    acc[k] = 0.0;
    const int q = threadIdx.x + k * kThreads;
    qi[k] = -2;
    qj[k] = 0;
    if (q == 0) {
      qi[k] = -1;
    } else if (q <= d) {
      qi[k] = q - 1;
      qj[k] = -1;
    } else if (q < Q) {
      const int t = q - 1 - d;
      int r = int((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while (tri(r + 1) <= t) ++r;
      while (tri(r) > t) --r;
      qi[k] = r;
      qj[k] = t - tri(r);
    }
  }
  __syncthreads();
  const int nchunks = (n + kChunk - 1) / kChunk;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int s0 = c * kChunk;
    const int cnt = min(kChunk, n - s0);
    for (int idx = threadIdx.x; idx < kChunk * d; idx += blockDim.x) {
      const int r = idx / d, j = idx % d;
      se[r][j] = r < cnt ? eps[size_t(s0 + r) * d + j] : 0.0;
      if (pathwise) sc[r][j] = r < cnt ? grad_z[size_t(s0 + r) * d + j] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < kChunk) {
      const int r = threadIdx.x;
      double f = 0.0;
      if (r < cnt) {
        double e2 = 0.0;
        for (int j = 0; j < d; ++j) e2 += se[r][j] * se[r][j];
        f = (-0.5 * e2 - s_logdet - 0.5 * d * kLn2Pi) - logp[s0 + r];
      }
      sf[r] = f;
    }
    __syncthreads();
    if (!pathwise) {
      for (int idx = threadIdx.x; idx < kChunk * d; idx += blockDim.x) {
        const int r = idx / d, j = idx % d;
        sc[r][j] = sf[r] * se[r][j];
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const int i = qi[k], j = qj[k];
      if (i == -2) continue;
      double a = 0.0;
      if (i == -1) {
        for (int r = 0; r < cnt; ++r) a += sf[r];
      } else if (j == -1) {
        for (int r = 0; r < cnt; ++r) a += sc[r][i];
      } else {
        for (int r = 0; r < cnt; ++r) a += sc[r][i] * se[r][j];
      }
      acc[k] += a;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kSlots; ++k) {
    const int q = threadIdx.x + k * kThreads;
    if (q < Q) partial[size_t(blockIdx.x) * Q + q] = acc[k];
  }
}

// Sum the blocks' moments, form the gradient in phi, optional Adam. One block.
__global__ void __launch_bounds__(kThreads) k_vi_finish(int n, int d, int nblk, const double* __restrict__ partial,
                                                        int pathwise, double* __restrict__ phi, double* __restrict__ m,
                                                        double* __restrict__ v, double c1, double c2, double lr,
                                                        double b1, double b2, double adam_eps,
                                                        double* __restrict__ grad_out, double* __restrict__ loss_out) {
  __shared__ double S[kMaxQ];
  __shared__ double L[GL_VI_MAX_D][GL_VI_MAX_D];
  __shared__ double E[GL_VI_MAX_D][GL_VI_MAX_D];   // symmetric second moment (score) / result rows
  __shared__ double a[GL_VI_MAX_D];
  const int Q = 1 + d + tri(d);
  const int P = d + tri(d);
  const double inv_n = 1.0 / double(n);
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += partial[size_t(b) * Q + q];
    S[q] = t * inv_n;
  }
  for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) {
    const int i = idx / d, j = idx % d;
    L[i][j] = j < i ? phi[d + tri(i) + j] : (j == i ? exp(phi[d + tri(i) + i]) : 0.0);
  }
  __syncthreads();
  const double fbar = S[0];
  if (threadIdx.x == 0) loss_out[0] = fbar;
  if (!pathwise) {
    for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) {
      const int i = idx / d, j = idx % d;
      E[i][j] = i >= j ? S[1 + d + tri(i) + j] : S[1 + d + tri(j) + i];
    }
    __syncthreads();
    // columns j = 0..d-1 of L^-T E (back substitution on L^T, rows d-1 down to j),
    // and column d: L^-T a with a = mean(f eps). One thread per column.
    if (threadIdx.x <= d) {
      const int j = threadIdx.x;
      double y[GL_VI_MAX_D];
      const int lo = j < d ? j : 0;
      for (int i = d - 1; i >= lo; --i) {
        double x = j < d ? E[i][j] : S[1 + i];
        for (int k = i + 1; k < d; ++k) x -= L[k][i] * y[k];
        y[i] = x / L[i][i];
      }
      if (j < d) {
        for (int i = j; i < d; ++i) E[i][j] = y[i];   // column j, rows >= j: read and written by this thread only
      } else {
        for (int i = 0; i < d; ++i) a[i] = y[i];
      }
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double g;
    if (p < d) {
      g = pathwise ? -S[1 + p] : a[p];
    } else {
      const int t = p - d;
      int i = int((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while (tri(i + 1) <= t) ++i;
      while (tri(i) > t) --i;
      const int j = t - tri(i);
      if (pathwise) {
        g = -S[1 + d + t];
        if (i == j) g = g * L[i][i] - 1.0;
      } else {
        g = E[i][j];
        if (i == j) g = (g - fbar / L[i][i]) * L[i][i];
      }
    }
    grad_out[p] = g;
    if (m) {
      const double mi = b1 * m[p] + (1.0 - b1) * g;
      const double vi = b2 * v[p] + (1.0 - b2) * g * g;
      m[p] = mi;
      v[p] = vi;
      phi[p] -= lr * (mi / c1) / (sqrt(vi / c2) + adam_eps);
    }
  }
}

// Sum the blocks' partial moments in block order: the moment sums of this
// call's draws (other processes' draws are added by the caller).
__global__ void k_vi_sum(int Q, int nblk, const double* __restrict__ partial, double* __restrict__ sums) {
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += partial[size_t(b) * Q + q];
    sums[q] = t;
  }
}

int finish(cudaStream_t st, const char* what) {
  cudaError_t e = gl_internal::hooks()->after(GL_K_OTHER, st);
  return e == cudaSuccess ? GL_OK : gl_internal::cuda_error(e, what);
}

}  // namespace

extern "C" {

size_t gl_vi_param_count(int d) { return (d < 1 || d > GL_VI_MAX_D) ? 0 : size_t(d) + size_t(tri(d)); }

size_t gl_vi_workspace_bytes(int n, int d) {
  if (n < 1 || d < 1 || d > GL_VI_MAX_D) return 0;
  return size_t(n_blocks(n)) * size_t(1 + d + tri(d)) * sizeof(double);
}

int gl_vi_sample(int n, int d, const double* eps, const double* phi, const gl_prior_entry* prior, double* z_out,
                 float* theta_out, void* stream) {
  if (n < 0 || d < 1 || d > GL_VI_MAX_D) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad n or d");
  if (prior && d != GL_NPARAM) return gl_internal::set_error(GL_ERR_INVALID_ARG, "a prior needs d == 22");
  PriorTable P{};
  if (prior) {
    int rc = load_table(prior, P);
    if (rc != GL_OK) return rc;
  }
  if (n == 0) return GL_OK;
  if (!eps || !phi || !z_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl_internal::hooks()->before(GL_K_OTHER, st);
  int g = (n + 3) / 4;
  g = g > 4096 ? 4096 : g;
  k_vi_sample<<<g, 128, 0, st>>>(n, d, eps, phi, z_out, theta_out, P, prior ? 1 : 0);
  return finish(st, "k_vi_sample");
}

int gl_vi_step(int n, int d, const double* eps, const double* logp, const double* grad_z, int estimator,
               double* phi, double* m, double* v, int t, double lr, double beta1, double beta2, double adam_eps,
               double* grad_out, double* loss_out, void* workspace, void* stream) {
  if (n < 1 || d < 1 || d > GL_VI_MAX_D) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad n or d");
  if (estimator != GL_VI_SCORE && estimator != GL_VI_PATHWISE)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "unknown estimator");
  if (!eps || !logp || !phi || !grad_out || !loss_out || !workspace ||
      (estimator == GL_VI_PATHWISE && !grad_z))
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if ((m == nullptr) != (v == nullptr)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "m and v: both or neither");
  if (m && (t < 1 || !std::isfinite(lr))) return gl_internal::set_error(GL_ERR_INVALID_ARG, "t < 1 or lr");
  const int nb = n_blocks(n);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl::Hooks* h = gl_internal::hooks();
  double* part = static_cast<double*>(workspace);
  const int pw = estimator == GL_VI_PATHWISE ? 1 : 0;
  h->before(GL_K_OTHER, st);
  k_vi_moments<<<nb, kThreads, 0, st>>>(n, d, eps, logp, grad_z, phi, pw, part);
  int rc = finish(st, "k_vi_moments");
  if (rc != GL_OK) return rc;
  const double c1 = m ? 1.0 - std::pow(beta1, t) : 1.0, c2 = m ? 1.0 - std::pow(beta2, t) : 1.0;
  h->before(GL_K_OTHER, st);
  k_vi_finish<<<1, kThreads, 0, st>>>(n, d, nb, part, pw, phi, m, v, c1, c2, lr, beta1, beta2, adam_eps, grad_out,
                                      loss_out);
  return finish(st, "k_vi_finish");
}

int gl_vi_moments(int n, int d, const double* eps, const double* logp, const double* grad_z, int estimator,
                  const double* phi, void* workspace, double* sums_out, void* stream) {
  if (n < 1 || d < 1 || d > GL_VI_MAX_D) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad n or d");
  if (estimator != GL_VI_SCORE && estimator != GL_VI_PATHWISE)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "unknown estimator");
  if (!eps || !logp || !phi || !workspace || !sums_out || (estimator == GL_VI_PATHWISE && !grad_z))
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  const int nb = n_blocks(n);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gl::Hooks* h = gl_internal::hooks();
  double* part = static_cast<double*>(workspace);
  h->before(GL_K_OTHER, st);
  k_vi_moments<<<nb, kThreads, 0, st>>>(n, d, eps, logp, grad_z, phi, estimator == GL_VI_PATHWISE ? 1 : 0, part);
  int rc = finish(st, "k_vi_moments");
  if (rc != GL_OK) return rc;
  h->before(GL_K_OTHER, st);
  k_vi_sum<<<1, kThreads, 0, st>>>(1 + d + tri(d), nb, part, sums_out);
  return finish(st, "k_vi_sum");
}

int gl_vi_apply(int n_total, int d, int nparts, const double* sums, int estimator, double* phi, double* m, double* v, int t,
                double lr, double beta1, double beta2, double adam_eps, double* grad_out, double* loss_out,
                void* stream) {
  if (n_total < 1 || d < 1 || d > GL_VI_MAX_D || nparts < 1)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad n, d or nparts");
  if (estimator != GL_VI_SCORE && estimator != GL_VI_PATHWISE)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "unknown estimator");
  if (!sums || !phi || !grad_out || !loss_out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null pointer");
  if ((m == nullptr) != (v == nullptr)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "m and v: both or neither");
  if (m && (t < 1 || !std::isfinite(lr))) return gl_internal::set_error(GL_ERR_INVALID_ARG, "t < 1 or lr");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double c1 = m ? 1.0 - std::pow(beta1, t) : 1.0, c2 = m ? 1.0 - std::pow(beta2, t) : 1.0;
  gl_internal::hooks()->before(GL_K_OTHER, st);
  k_vi_finish<<<1, kThreads, 0, st>>>(n_total, d, nparts, sums, estimator == GL_VI_PATHWISE ? 1 : 0, phi, m, v, c1, c2,
                                      lr, beta1, beta2, adam_eps, grad_out, loss_out);
  return finish(st, "k_vi_finish");
}

}  // extern "C"
