// gl_variant.cu - the likelihood with the observed-image variance of
// arXiv:2202.07663, Sec. 2.1.2 (sigma_tot^2 = sigma_bkg^2 + I_obs/(G t_exp),
// negative observed pixels counted as zero), profiled over the two light
// amplitudes. With a parameter-independent variance the model is linear in
// (I_l, I_s), M = I_l A_l + I_s A_s, and the amplitudes maximising log L solve
//   [<A_l,A_l> <A_l,A_s>; <A_s,A_l> <A_s,A_s>] [I_l; I_s] = [<A_l,D>; <A_s,D>],
// <a,b> = sum_pixels a b / sigma_tot^2. The basis images A come from the
// simulation path at unit amplitudes (one ray pass for both, k_ray_fwd_basis);
// these kernels reduce and solve the 2x2 systems (FP64), evaluate log L and
// d log L / d M of the profiled model, and zero the amplitude entries of the
// profiled gradient.
#include <cuda_runtime.h>

#include "gl_internal.h"

namespace {

constexpr int kIL = 14, kIS = 21;
constexpr double kSingular = 1e-12;   // relative size below which a self-product or det counts as zero
constexpr int kSolveThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += sh[i];
  return t;   // valid in thread 0
}

// One block per vector: the five weighted inner products, the 2x2 solve, the
// amplitudes (FP64) and the parameter row with the amplitudes substituted;
// then, with loglik set, the model M = I_l A_l + I_s A_s (the PSF convolution
// is linear, so the convolved basis images give the convolved model), log L
// and chi^2 (FP32 per pixel and thread, FP64 across threads) and, with dldm
// set, d log L / d M per pixel into dldm[b] (the next pass correlates it with
// the PSF for the gradient).
__global__ void __launch_bounds__(kSolveThreads) k_amp_solve(int B, int HW, const float* __restrict__ images,
                                                             const float* __restrict__ data,
                                                             const float* __restrict__ sigma2,
                                                             const float* __restrict__ params,
                                                             float* __restrict__ params_out,
                                                             double* __restrict__ amps, float inv_gain,
                                                             double* __restrict__ loglik,
                                                             double* __restrict__ chi2, float* __restrict__ dldm) {
  __shared__ double sh[kSolveThreads / 32];
  __shared__ double s_amp[2];
  const int b = blockIdx.x;
  if (b >= B) return;
  const float* Al = images + size_t(2 * b) * HW;
  const float* As = images + size_t(2 * b + 1) * HW;
  double gll = 0.0, gls = 0.0, gss = 0.0, rl = 0.0, rs = 0.0;
  for (int i = threadIdx.x; i < HW; i += blockDim.x) {
    const double w = 1.0 / double(sigma2[i]);
    const double al = Al[i], as = As[i], d = data[i];
    gll += w * al * al;
    gls += w * al * as;
    gss += w * as * as;
    rl += w * al * d;
    rs += w * as * d;
  }
  gll = block_sum(gll, sh);
  gls = block_sum(gls, sh);
  gss = block_sum(gss, sh);
  rl = block_sum(rl, sh);
  rs = block_sum(rs, sh);
  if (threadIdx.x == 0) {
    double il = 0.0, is = 0.0;
    const double gmax = fmax(gll, gss);
    const bool live_l = gll > kSingular * gmax, live_s = gss > kSingular * gmax;
    const double det = gll * gss - gls * gls;
    if (live_l && live_s && det > kSingular * gll * gss) {
      il = (gss * rl - gls * rs) / det;
      is = (gll * rs - gls * rl) / det;
    } else if (live_l || live_s) {
      if (live_l && (!live_s || gll >= gss)) {
        il = rl / gll;
      } else {
        is = rs / gss;
      }
    }
    amps[2 * b] = il;
    amps[2 * b + 1] = is;
    s_amp[0] = il;
    s_amp[1] = is;
  }
  for (int j = threadIdx.x; j < gl::NPARAM; j += blockDim.x) {
    // thread 0 wrote amps above; the other rows are copies of the input
    if (j != kIL && j != kIS) params_out[size_t(b) * gl::NPARAM + j] = params[size_t(b) * gl::NPARAM + j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    params_out[size_t(b) * gl::NPARAM + kIL] = float(s_amp[0]);
    params_out[size_t(b) * gl::NPARAM + kIS] = float(s_amp[1]);
  }
  if (!loglik) return;
  // the amplitudes as the model evaluation uses them (the substituted FP32 row)
  const float il = float(s_amp[0]), is = float(s_amp[1]);
  float ll = 0.f, c2 = 0.f;
  for (int i = threadIdx.x; i < HW; i += blockDim.x) {
    const float M = fmaf(il, Al[i], is * As[i]);
    const float v = fmaf(M, inv_gain, sigma2[i]);
    const float res = data[i] - M;
    const float iv = 1.0f / v;
    const float t2 = res * res * iv;
    c2 += t2;
    ll += t2 + logf(6.28318530717958648f * v);
    // d log L / d M = res/v + (res^2/v^2 - 1/v) / (2 G t_exp)
    if (dldm) dldm[size_t(b) * HW + i] = fmaf(0.5f * inv_gain, fmaf(t2, iv, -iv), res * iv);
  }
  const double L = block_sum(double(ll), sh);
  const double C = block_sum(double(c2), sh);
  if (threadIdx.x == 0) {
    loglik[b] = -0.5 * L;
    if (chi2) chi2[b] = C;
  }
}

__global__ void k_zero_amp_grad(int B, double* __restrict__ grad) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    grad[size_t(b) * gl::NPARAM + kIL] = 0.0;
    grad[size_t(b) * gl::NPARAM + kIS] = 0.0;
  }
}

int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return int(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

namespace gl_internal {

cudaError_t launch_amp_solve(int B, int HW, const float* images, const float* data, const float* sigma2,
                             const float* params, float* params_out, double* amps, float inv_gain, double* loglik,
                             double* chi2, float* dldm, cudaStream_t st) {
  hooks()->before(GL_K_OTHER, st);
  k_amp_solve<<<B, kSolveThreads, 0, st>>>(B, HW, images, data, sigma2, params, params_out, amps, inv_gain, loglik,
                                           chi2, dldm);
  return hooks()->after(GL_K_OTHER, st);
}

cudaError_t launch_zero_amp_grad(int B, double* grad, cudaStream_t st) {
  hooks()->before(GL_K_OTHER, st);
  k_zero_amp_grad<<<grid_for(B, 128), 128, 0, st>>>(B, grad);
  return hooks()->after(GL_K_OTHER, st);
}

}  // namespace gl_internal
