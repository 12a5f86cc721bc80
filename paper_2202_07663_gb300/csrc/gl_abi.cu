// gl_abi.cu - C ABI of the batched lens likelihood (declarations and the
// contract of every entry point are in include/gigalens.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "gl_device.cuh"
#include "gl_internal.h"
#include "gl_launch.h"

using gl::Seg;
using gl::VecConst;

struct gl_system {
  int device = 0;
  int H = 0, W = 0, K = 0, k = 1;
  double pixel_scale = 0.0, gain_exposure = 0.0;
  float* d_image = nullptr;
  float* d_sigma2 = nullptr;
  float* d_psf = nullptr;
  // the PSF as psf_rank separable terms (0: convolve with the K x K PSF directly)
  int psf_rank = 0;
  float* d_psf_sep = nullptr;   // [psf_rank][2][K]: sigma_r u_r (rows), v_r (columns)
  // scratch, grown on demand
  long long cap_B = 0;
  long long cap_partial = 0;   // doubles
  VecConst* d_vc = nullptr;
  float* d_work = nullptr;
  double* d_partial = nullptr;
  // device staging of the host-buffer entry point
  long long cap_host = 0;
  float* d_params = nullptr;
  double* d_ll = nullptr;
  double* d_c2 = nullptr;
  double* d_grad = nullptr;
  // likelihood profiled over the light amplitudes: basis parameter rows and
  // images (2 per vector), parameter rows with the solved amplitudes
  long long cap_prof = 0;
  float* d_pimg = nullptr;
  float* d_pfull = nullptr;
  double* d_pamps = nullptr;
};

namespace {

thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error of this thread, if any
  if (e == cudaErrorMemoryAllocation) return fail(GL_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(GL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GL_CUDA(call, what)                  \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// ------------------------------------------------------- instrumentation --

std::atomic<long long> g_launches{0};

struct Profiler final : gl::Hooks {
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::mutex mu;
  bool on = false;
  unsigned kinds = ~0u;   // the kernel kinds bracketed while on (bit k: kind k)
  bool rec_cur = false;
  std::vector<Rec> recs;
  Rec cur{};
  long long launches[GL_KERNEL_KINDS] = {};
  double ms[GL_KERNEL_KINDS] = {};

  void before(int kind, cudaStream_t st) override {
    rec_cur = on && (kinds >> kind & 1u);
    if (!rec_cur) return;
    cur.kind = kind;
    cudaEventCreate(&cur.a);
    cudaEventCreate(&cur.b);
    cudaEventRecord(cur.a, st);
  }
  cudaError_t after(int kind, cudaStream_t st) override {
    (void)kind;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (rec_cur) {
      cudaEventRecord(cur.b, st);
      std::lock_guard<std::mutex> lk(mu);
      recs.push_back(cur);
      rec_cur = false;
    }
    return e;
  }
  void drain() {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& r : recs) {
      float t = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.kind] += t;
        launches[r.kind] += 1;
      }
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    recs.clear();
  }
};

Profiler g_prof;

// ------------------------------------------------------------ helpers ----

bool finite_all(const float* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

int max_smem_optin(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// The PSF P (K x K, row-major, FP64 values of the floats the device uses) as
// a sum of separable terms P = sum_r sigma_r u_r v_r^T, from its singular
// value decomposition by one-sided Jacobi rotations (Hestenes 1958): the
// columns of A = P are rotated pairwise until orthogonal, A V = U Sigma.
// The rank kept is the smallest whose dropped singular values have a root
// sum of squares of at most 2^-24 ||P||_F: no more than the rounding that
// the PSF's FP32 values already carry (half an ulp, 2^-24 relative, in every
// entry), so that a PSF which is separable before rounding stays so. The
// factors are used only if 2 R K <= K^2 / 2 (then two 1-D passes per term
// are at least twice as cheap as the 2-D pass). Returns R (0: keep the
// 2-D convolution) and fac = [R][2][K] as floats: sigma_r u_r, then v_r.
int psf_separable(const std::vector<float>& psf, int K, std::vector<float>& fac) {
  const int n = K;
  std::vector<double> A(size_t(n) * n), V(size_t(n) * n, 0.0);
  for (int i = 0; i < n * n; ++i) A[i] = psf[i];
  for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < n; ++i) {
          const double ap = A[size_t(i) * n + p], aq = A[size_t(i) * n + q];
          alpha += ap * ap;
          beta += aq * aq;
          gamma += ap * aq;
        }
        if (gamma == 0.0 || std::fabs(gamma) <= 1e-17 * std::sqrt(alpha * beta)) continue;
        off = std::fmax(off, std::fabs(gamma) / std::sqrt(alpha * beta));
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < n; ++i) {
          double& ap = A[size_t(i) * n + p];
          double& aq = A[size_t(i) * n + q];
          const double x = ap, y = aq;
          ap = c * x - sn * y;
          aq = sn * x + c * y;
          double& vp = V[size_t(i) * n + p];
          double& vq = V[size_t(i) * n + q];
          const double vx = vp, vy = vq;
          vp = c * vx - sn * vy;
          vq = sn * vx + c * vy;
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<std::pair<double, int>> sv(n);
  double total = 0.0;
  for (int j = 0; j < n; ++j) {
    double s2 = 0.0;
    for (int i = 0; i < n; ++i) s2 += A[size_t(i) * n + j] * A[size_t(i) * n + j];
    sv[j] = {std::sqrt(s2), j};
    total += s2;
  }
  std::sort(sv.begin(), sv.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
    return a.first > b.first;
  });
  int R = n;
  double tail = 0.0;   // sum of the squares of the dropped singular values
  const double tol2 = 0x1p-48;   // (2^-24)^2
  while (R > 1 && tail + sv[R - 1].first * sv[R - 1].first <= tol2 * total) {
    tail += sv[R - 1].first * sv[R - 1].first;
    --R;
  }
  if (!(total > 0.0) || 4 * R > K) return 0;
  fac.assign(size_t(R) * 2 * n, 0.f);
  for (int r = 0; r < R; ++r) {
    const int j = sv[r].second;
    for (int i = 0; i < n; ++i) {
      fac[(size_t(r) * 2) * n + i] = float(A[size_t(i) * n + j]);         // sigma_r u_r (column j of A V)
      fac[(size_t(r) * 2 + 1) * n + i] = float(V[size_t(i) * n + j]);     // v_r (column j of V)
    }
  }
  return R;
}

// Static shared memory of the convolution kernel besides the image (Seg + reductions), with margin.
constexpr size_t CONV_STATIC_SMEM = 2048;

int ensure_scratch(gl_system* s, long long B, long long partial) {
  if (B > s->cap_B) {
    cudaFree(s->d_vc);
    cudaFree(s->d_work);
    s->d_vc = nullptr;
    s->d_work = nullptr;
    s->cap_B = 0;
    GL_CUDA(cudaMalloc(&s->d_vc, sizeof(VecConst) * size_t(B)), "scratch (vector constants)");
    GL_CUDA(cudaMalloc(&s->d_work, sizeof(float) * size_t(B) * s->H * s->W), "scratch (image work)");
    s->cap_B = B;
  }
  if (partial > s->cap_partial) {
    cudaFree(s->d_partial);
    s->d_partial = nullptr;
    s->cap_partial = 0;
    GL_CUDA(cudaMalloc(&s->d_partial, sizeof(double) * size_t(partial)), "scratch (partials)");
    s->cap_partial = partial;
  }
  return GL_OK;
}

void partial_need(const gl_system* s, int B, int* ntiles, int* tile_pix, long long* partial) {
  gl::plan_tiles(B, s->H, s->W, s->k, ntiles, tile_pix);
  *partial = (long long)B * (*ntiles) * gl::NACC;
}

Seg make_seg(const gl_system* s, const float* params, int B) {
  Seg g;
  std::memset(&g, 0, sizeof(g));
  g.image = s->d_image;
  g.sigma2 = s->d_sigma2;
  g.psf = s->d_psf;
  g.psf_sep = s->d_psf_sep;
  g.psf_rank = s->psf_rank;
  g.H = s->H;
  g.W = s->W;
  g.K = s->K;
  g.k = s->k;
  // subpixel centres at (j - (kW - 1)/2) pixel_scale/k = (2j + 1 - kW) h, h = pixel_scale/(2k)
  const double h = s->pixel_scale / (2.0 * s->k);
  g.hh = float(h);
  g.hl = float(h - double(g.hh));
  g.nx0 = 1 - s->k * s->W;
  g.ny0 = 1 - s->k * s->H;
  g.inv_gain = s->gain_exposure > 0.0 ? float(1.0 / s->gain_exposure) : 0.f;
  g.params = params;
  g.B = B;
  gl::plan_tiles(B, s->H, s->W, s->k, &g.ntiles, &g.tile_pix);
  g.vc = s->d_vc;
  g.work = s->d_work;
  g.partial = s->d_partial;
  g.conv_two_buf = gl::conv_two_buf(s->H, s->W, s->K) ? 1 : 0;
  g.conv_sep = gl::conv_sep_ok(s->H, s->W, s->K, s->psf_rank) ? 1 : 0;
  return g;
}

// A system's data and scratch live on the device that was current when it was
// created; a call made with another device current would launch there on
// pointers of the first one. Refused, not switched: the caller owns the
// current device and the stream, which belongs to one device.
int check_device(const gl_system* s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != s->device)
    return fail(GL_ERR_INVALID_ARG, "the system lives on device %d but device %d is current", s->device, dev);
  return GL_OK;
}

int check_call(const gl_system* s, const float* params, int B) {
  if (!s) return fail(GL_ERR_INVALID_ARG, "null gl_system");
  if (B < 0 || B > (1 << 24)) return fail(GL_ERR_INVALID_ARG, "B = %d outside [0, 2^24]", B);
  if (B > 0 && !params) return fail(GL_ERR_INVALID_ARG, "null params");
  return check_device(s);
}

int run_one(gl_system* s, const float* params, int B, double* ll, double* c2, double* grad, float* sim, int mode,
            cudaStream_t st) {
  int ntiles, tile_pix;
  long long partial;
  partial_need(s, B, &ntiles, &tile_pix, &partial);
  int rc = ensure_scratch(s, B, partial);
  if (rc != GL_OK) return rc;
  Seg g = make_seg(s, params, B);
  g.loglik = ll;
  g.chi2 = c2;
  g.grad = grad;
  g.sim = sim;
  cudaError_t e = gl::launch_one(g, mode, st, &g_prof);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return GL_OK;
}

}  // namespace

// Internal helpers for other translation units of the library (not ABI).
namespace gl_internal {

int system_device_check(const gl_system* s) { return check_device(s); }

size_t scratch_held(const gl_system* s) {
  return sizeof(VecConst) * size_t(s->cap_B) + sizeof(float) * size_t(s->cap_B) * s->H * s->W +
         sizeof(double) * size_t(s->cap_partial);
}

// Segment of a call on sys with every scratch pointer left null.
gl::Seg seg_without_scratch(const gl_system* s, const float* params, int B) {
  Seg g = make_seg(s, params, B);
  g.vc = nullptr;
  g.work = nullptr;
  g.partial = nullptr;
  return g;
}

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

int cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

gl::Hooks* hooks() { return &g_prof; }

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace gl_internal

namespace {

// Shared by the two constructors: validated sizes, the per-pixel variance s2.
int create_impl(gl_system** out, const float* image, const std::vector<float>& s2, int H, int W, const float* psf,
                int K, double pixel_scale, int supersample, double gain_exposure, void* stream) {
  const size_t n = size_t(H) * W;
  int dev = 0;
  GL_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  const size_t smem = gl::conv_smem_bytes(H, W, K, false) + CONV_STATIC_SMEM;
  if (smem > size_t(max_smem_optin(dev)))
    return fail(GL_ERR_UNSUPPORTED, "padded %dx%d image with K=%d needs %zu B of shared memory (> %d)", H, W, K,
                smem, max_smem_optin(dev));
  // A detector pixel records the flux falling on it: the mean surface brightness
  // over its subpixels times the pixel area. The convolution is linear, so the
  // area is folded into the PSF weights once here.
  const double area = pixel_scale * pixel_scale;
  std::vector<float> psf_area(size_t(K) * K);
  for (size_t i = 0; i < psf_area.size(); ++i) psf_area[i] = float(double(psf[i]) * area);
  gl_system* s = new gl_system();
  s->device = dev;
  s->H = H;
  s->W = W;
  s->K = K;
  s->k = supersample;
  s->pixel_scale = pixel_scale;
  s->gain_exposure = gain_exposure;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaMalloc(&s->d_image, n * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_sigma2, n * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_psf, size_t(K) * K * sizeof(float))) != cudaSuccess ||
      (e = cudaMemcpyAsync(s->d_image, image, n * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s->d_sigma2, s2.data(), n * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s->d_psf, psf_area.data(), size_t(K) * K * sizeof(float), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    gl_system_destroy(s);
    return cuda_fail(e, "gl_system_create upload");
  }
  std::vector<float> fac;
  const int R = psf_separable(psf_area, K, fac);
  if (R > 0 && gl::conv_sep_any(H, W, K, R)) {   // factors kept only where the 1-D passes run
    if ((e = cudaMalloc(&s->d_psf_sep, fac.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMemcpy(s->d_psf_sep, fac.data(), fac.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
      gl_system_destroy(s);
      return cuda_fail(e, "gl_system_create upload (PSF factors)");
    }
    s->psf_rank = R;
  }
  *out = s;
  return GL_OK;
}

int check_create(gl_system** out, const float* image, int H, int W, const float* psf, int K, double pixel_scale,
                 int supersample, double gain_exposure) {
  if (!out) return fail(GL_ERR_INVALID_ARG, "null out");
  *out = nullptr;
  if (!image || !psf) return fail(GL_ERR_INVALID_ARG, "null image or psf");
  if (H < 1 || W < 1 || H > 4096 || W > 4096) return fail(GL_ERR_INVALID_ARG, "image size %dx%d", H, W);
  if (K < 1 || K > 63 || (K % 2) == 0) return fail(GL_ERR_INVALID_ARG, "PSF side K = %d must be odd in [1, 63]", K);
  if (!(pixel_scale > 0.0) || !std::isfinite(pixel_scale))
    return fail(GL_ERR_INVALID_ARG, "pixel_scale must be > 0");
  if (supersample < 1 || supersample > 16) return fail(GL_ERR_INVALID_ARG, "supersample = %d", supersample);
  if (!std::isfinite(gain_exposure)) return fail(GL_ERR_INVALID_ARG, "gain_exposure not finite");
  if (!finite_all(image, size_t(H) * W)) return fail(GL_ERR_INVALID_ARG, "image has non-finite values");
  if (!finite_all(psf, size_t(K) * K)) return fail(GL_ERR_INVALID_ARG, "psf has non-finite values");
  return GL_OK;
}

// The background variance per pixel from a noise map or a scalar.
int background_variance(const float* noise_map, float sigma_bkg, size_t n, std::vector<float>& s2) {
  s2.resize(n);
  if (noise_map) {
    for (size_t i = 0; i < n; ++i) {
      if (!(noise_map[i] > 0.f) || !std::isfinite(noise_map[i]))
        return fail(GL_ERR_INVALID_ARG, "noise_map[%zu] must be finite and > 0", i);
      s2[i] = noise_map[i] * noise_map[i];
    }
  } else {
    if (!(sigma_bkg > 0.f) || !std::isfinite(sigma_bkg)) return fail(GL_ERR_INVALID_ARG, "sigma_bkg must be > 0");
    for (size_t i = 0; i < n; ++i) s2[i] = sigma_bkg * sigma_bkg;
  }
  return GL_OK;
}

}  // namespace

extern "C" {

int gl_system_create(gl_system** out, const float* image, const float* noise_map, float sigma_bkg, int H, int W,
                     const float* psf, int K, double pixel_scale, int supersample, double gain_exposure,
                     void* stream) {
  int rc = check_create(out, image, H, W, psf, K, pixel_scale, supersample, gain_exposure);
  if (rc != GL_OK) return rc;
  std::vector<float> s2;
  rc = background_variance(noise_map, sigma_bkg, size_t(H) * W, s2);
  if (rc != GL_OK) return rc;
  return create_impl(out, image, s2, H, W, psf, K, pixel_scale, supersample, gain_exposure, stream);
}

int gl_system_create_obsvar(gl_system** out, const float* image, const float* noise_map, float sigma_bkg, int H,
                            int W, const float* psf, int K, double pixel_scale, int supersample,
                            double gain_exposure, void* stream) {
  int rc = check_create(out, image, H, W, psf, K, pixel_scale, supersample, gain_exposure);
  if (rc != GL_OK) return rc;
  std::vector<float> s2;
  rc = background_variance(noise_map, sigma_bkg, size_t(H) * W, s2);
  if (rc != GL_OK) return rc;
  if (gain_exposure > 0.0)
    for (size_t i = 0; i < s2.size(); ++i)
      s2[i] = float(double(s2[i]) + (image[i] > 0.f ? double(image[i]) : 0.0) / gain_exposure);
  return create_impl(out, image, s2, H, W, psf, K, pixel_scale, supersample, 0.0, stream);
}

int gl_system_destroy(gl_system* s) {
  if (!s) return GL_OK;
  // free on the system's own device, then give the caller's current device back
  int cur = s->device;
  cudaGetDevice(&cur);
  if (cur != s->device) cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  cudaFree(s->d_image);
  cudaFree(s->d_sigma2);
  cudaFree(s->d_psf);
  cudaFree(s->d_psf_sep);
  cudaFree(s->d_vc);
  cudaFree(s->d_work);
  cudaFree(s->d_partial);
  cudaFree(s->d_params);
  cudaFree(s->d_ll);
  cudaFree(s->d_c2);
  cudaFree(s->d_grad);
  cudaFree(s->d_pimg);
  cudaFree(s->d_pfull);
  cudaFree(s->d_pamps);
  const int dev = s->device;
  delete s;
  if (cur != dev) cudaSetDevice(cur);
  return GL_OK;
}

size_t gl_system_scratch_bytes(const gl_system* s, int B) {
  if (!s || B < 0) return 0;
  int ntiles, tile_pix;
  long long partial;
  partial_need(s, B, &ntiles, &tile_pix, &partial);
  return sizeof(VecConst) * size_t(B) + sizeof(float) * size_t(B) * s->H * s->W + sizeof(double) * size_t(partial);
}

size_t gl_system_scratch_held(const gl_system* s) { return s ? gl_internal::scratch_held(s) : 0; }

size_t gl_system_resident_bytes(const gl_system* s) {
  if (!s) return 0;
  return sizeof(float) * (2 * size_t(s->H) * s->W + size_t(s->K) * s->K + 2 * size_t(s->psf_rank) * s->K);
}

int gl_system_psf_rank(const gl_system* s) {
  if (!s) return fail(GL_ERR_INVALID_ARG, "null gl_system");
  return s->psf_rank;
}

int gl_psf_factor(const float* psf, int K, float* fac, int fac_len, int* rank) {
  if (!psf || !rank) return fail(GL_ERR_INVALID_ARG, "null psf or rank");
  if (K < 1 || K % 2 == 0 || K > 255) return fail(GL_ERR_INVALID_ARG, "K = %d (odd, 1..255)", K);
  std::vector<float> p(psf, psf + size_t(K) * K), f;
  for (float v : p)
    if (!std::isfinite(v)) return fail(GL_ERR_INVALID_ARG, "non-finite PSF value");
  const int R = psf_separable(p, K, f);
  if (fac && R > 0) {
    if (fac_len < 2 * R * K) return fail(GL_ERR_INVALID_ARG, "fac holds %d floats, %d needed", fac_len, 2 * R * K);
    std::copy(f.begin(), f.end(), fac);
  }
  *rank = R;
  return GL_OK;
}

int gl_system_reserve(gl_system* s, int B) {
  if (!s) return fail(GL_ERR_INVALID_ARG, "null gl_system");
  if (B < 0 || B > (1 << 24)) return fail(GL_ERR_INVALID_ARG, "B = %d", B);
  int rc = check_device(s);
  if (rc != GL_OK) return rc;
  // partial need is largest at small B (more tiles per vector); take the max over B' <= B
  long long need = 0;
  for (int b : {1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, B}) {
    if (b > B || b < 1) continue;
    int nt, tp;
    long long p;
    partial_need(s, b, &nt, &tp, &p);
    need = p > need ? p : need;
  }
  return ensure_scratch(s, B, need);
}

int gl_loglik(gl_system* s, const float* params, int B, double* loglik_out, double* chi2_out, void* stream) {
  int rc = check_call(s, params, B);
  if (rc != GL_OK) return rc;
  if (B == 0) return GL_OK;
  if (!loglik_out) return fail(GL_ERR_INVALID_ARG, "null loglik_out");
  return run_one(s, params, B, loglik_out, chi2_out, nullptr, nullptr, gl::MODE_LOGLIK,
                 static_cast<cudaStream_t>(stream));
}

int gl_loglik_grad(gl_system* s, const float* params, int B, double* loglik_out, double* chi2_out, double* grad_out,
                   void* stream) {
  int rc = check_call(s, params, B);
  if (rc != GL_OK) return rc;
  if (B == 0) return GL_OK;
  if (!loglik_out || !grad_out) return fail(GL_ERR_INVALID_ARG, "null loglik_out or grad_out");
  return run_one(s, params, B, loglik_out, chi2_out, grad_out, nullptr, gl::MODE_GRAD,
                 static_cast<cudaStream_t>(stream));
}

int gl_simulate(gl_system* s, const float* params, int B, float* images_out, void* stream) {
  int rc = check_call(s, params, B);
  if (rc != GL_OK) return rc;
  if (B == 0) return GL_OK;
  if (!images_out) return fail(GL_ERR_INVALID_ARG, "null images_out");
  return run_one(s, params, B, nullptr, nullptr, nullptr, images_out, gl::MODE_SIM,
                 static_cast<cudaStream_t>(stream));
}

int gl_loglik_grad_profiled(gl_system* s, const float* params, int B, double* loglik_out, double* chi2_out,
                            double* grad_out, double* amps_out, void* stream) {
  int rc = check_call(s, params, B);
  if (rc != GL_OK) return rc;
  if (B == 0) return GL_OK;
  if (!loglik_out) return fail(GL_ERR_INVALID_ARG, "null loglik_out");
  if (s->gain_exposure > 0.0)
    return fail(GL_ERR_INVALID_ARG, "profiling the amplitudes needs a parameter-independent variance "
                                    "(gl_system_create_obsvar, or gain_exposure <= 0)");
  if (B > (1 << 23)) return fail(GL_ERR_INVALID_ARG, "B = %d: the basis images take 2B vectors", B);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B > s->cap_prof) {
    cudaFree(s->d_pimg);
    cudaFree(s->d_pfull);
    cudaFree(s->d_pamps);
    s->d_pimg = s->d_pfull = nullptr;
    s->d_pamps = nullptr;
    s->cap_prof = 0;
    const size_t hw = size_t(s->H) * s->W;
    GL_CUDA(cudaMalloc(&s->d_pimg, size_t(2) * B * hw * sizeof(float)), "profile scratch");
    GL_CUDA(cudaMalloc(&s->d_pfull, size_t(B) * GL_NPARAM * sizeof(float)), "profile scratch");
    GL_CUDA(cudaMalloc(&s->d_pamps, size_t(2) * B * sizeof(double)), "profile scratch");
    s->cap_prof = B;
  }
  double* amps = amps_out ? amps_out : s->d_pamps;
  // the two convolved unit-amplitude basis images of every vector (one ray
  // pass, 2B convolutions); the image scratch gets 2B slots, so the B-vector
  // pass below keeps it
  int ntiles, tile_pix;
  long long partial;
  partial_need(s, B, &ntiles, &tile_pix, &partial);
  rc = ensure_scratch(s, 2LL * B, partial);
  if (rc != GL_OK) return rc;
  Seg g = make_seg(s, params, B);
  g.sim = s->d_pimg;
  cudaError_t e = gl::launch_basis(g, st, &g_prof);
  if (e != cudaSuccess) return cuda_fail(e, "basis images");
  // amplitudes, then log L of M = I_l A_l + I_s A_s and d log L / d M into the
  // image scratch, which the correlation-only pass turns into the gradient
  const float inv_gain = s->gain_exposure > 0.0 ? float(1.0 / s->gain_exposure) : 0.f;
  e = gl_internal::launch_amp_solve(B, s->H * s->W, s->d_pimg, s->d_image, s->d_sigma2, params, s->d_pfull, amps,
                                    inv_gain, loglik_out, chi2_out, grad_out ? s->d_work : nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "k_amp_solve");
  if (!grad_out) return GL_OK;
  rc = run_one(s, s->d_pfull, B, nullptr, nullptr, grad_out, nullptr, gl::MODE_CORR, st);
  if (rc != GL_OK) return rc;
  e = gl_internal::launch_zero_amp_grad(B, grad_out, st);
  if (e != cudaSuccess) return cuda_fail(e, "k_zero_amp_grad");
  return GL_OK;
}

int gl_loglik_grad_host(gl_system* s, const float* params, int B, double* loglik_out, double* chi2_out,
                        double* grad_out, void* stream) {
  int rc = check_call(s, params, B);
  if (rc != GL_OK) return rc;
  if (B == 0) return GL_OK;
  if (!loglik_out || !grad_out) return fail(GL_ERR_INVALID_ARG, "null loglik_out or grad_out");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B > s->cap_host) {
    cudaFree(s->d_params);
    cudaFree(s->d_ll);
    cudaFree(s->d_c2);
    cudaFree(s->d_grad);
    s->d_params = nullptr;
    s->d_ll = s->d_c2 = s->d_grad = nullptr;
    s->cap_host = 0;
    GL_CUDA(cudaMalloc(&s->d_params, sizeof(float) * size_t(B) * GL_NPARAM), "host staging");
    GL_CUDA(cudaMalloc(&s->d_ll, sizeof(double) * size_t(B)), "host staging");
    GL_CUDA(cudaMalloc(&s->d_c2, sizeof(double) * size_t(B)), "host staging");
    GL_CUDA(cudaMalloc(&s->d_grad, sizeof(double) * size_t(B) * GL_NPARAM), "host staging");
    s->cap_host = B;
  }
  GL_CUDA(cudaMemcpyAsync(s->d_params, params, sizeof(float) * size_t(B) * GL_NPARAM, cudaMemcpyHostToDevice, st),
          "params upload");
  rc = run_one(s, s->d_params, B, s->d_ll, s->d_c2, s->d_grad, nullptr, gl::MODE_GRAD, st);
  if (rc != GL_OK) return rc;
  GL_CUDA(cudaMemcpyAsync(loglik_out, s->d_ll, sizeof(double) * size_t(B), cudaMemcpyDeviceToHost, st),
          "loglik download");
  if (chi2_out)
    GL_CUDA(cudaMemcpyAsync(chi2_out, s->d_c2, sizeof(double) * size_t(B), cudaMemcpyDeviceToHost, st),
            "chi2 download");
  GL_CUDA(cudaMemcpyAsync(grad_out, s->d_grad, sizeof(double) * size_t(B) * GL_NPARAM, cudaMemcpyDeviceToHost, st),
          "grad download");
  GL_CUDA(cudaStreamSynchronize(st), "stream synchronize");
  return GL_OK;
}

int gl_loglik_grad_grouped(gl_system* const* systems, const float* const* params, const int* B,
                           double* const* loglik_out, double* const* chi2_out, double* const* grad_out, int n,
                           void* stream) {
  if (n < 1 || n > GL_MAX_SEGMENTS) return fail(GL_ERR_INVALID_ARG, "n = %d segments", n);
  if (!systems || !params || !B || !loglik_out) return fail(GL_ERR_INVALID_ARG, "null array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<Seg> by_class[gl::CONV_CLASSES];
  bool any_grad = false, all_grad = true;
  for (int i = 0; i < n; ++i) {
    gl_system* s = systems[i];
    int rc = check_call(s, params[i], B[i]);
    if (rc != GL_OK) return rc;
    for (int j = 0; j < i; ++j)
      if (systems[j] == s) return fail(GL_ERR_INVALID_ARG, "system of segment %d repeats segment %d", i, j);
    if (B[i] == 0) continue;
    if (!loglik_out[i]) return fail(GL_ERR_INVALID_ARG, "null loglik_out[%d]", i);
    const bool g = grad_out && grad_out[i];
    any_grad = any_grad || g;
    all_grad = all_grad && g;
    int ntiles, tile_pix;
    long long partial;
    partial_need(s, B[i], &ntiles, &tile_pix, &partial);
    rc = ensure_scratch(s, B[i], partial);
    if (rc != GL_OK) return rc;
    Seg sg = make_seg(s, params[i], B[i]);
    sg.loglik = loglik_out[i];
    sg.chi2 = chi2_out ? chi2_out[i] : nullptr;
    sg.grad = g ? grad_out[i] : nullptr;
    by_class[gl::conv_class(s->K)].push_back(sg);
  }
  if (any_grad && !all_grad) return fail(GL_ERR_INVALID_ARG, "grad_out must be given for all segments or none");
  // table sorted by convolution class; item offsets in every item space
  std::vector<Seg> segs;
  std::vector<gl::ConvRun> runs;
  int vec_total = 0, ray_total = 0;
  for (int c = 0; c < gl::CONV_CLASSES; ++c) {
    if (by_class[c].empty()) continue;
    gl::ConvRun r{c, int(segs.size()), int(by_class[c].size()), 0, 0};
    for (Seg& sg : by_class[c]) {
      sg.vec_begin = vec_total;
      sg.ray_begin = ray_total;
      sg.conv_begin = r.nitems;
      vec_total += sg.B;
      ray_total += sg.B * sg.ntiles;
      r.nitems += sg.B;
      const size_t sm = gl::seg_conv_smem(sg);
      r.smem = sm > r.smem ? sm : r.smem;
      segs.push_back(sg);
    }
    runs.push_back(r);
  }
  if (segs.empty()) return GL_OK;
  Seg* d = nullptr;
  const size_t bytes = sizeof(Seg) * segs.size();
  GL_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), bytes, st), "segment table");
  cudaError_t e = cudaMemcpyAsync(d, segs.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = gl::launch_table(d, int(segs.size()), vec_total, ray_total, runs.data(), int(runs.size()),
                         all_grad ? gl::MODE_GRAD : gl::MODE_LOGLIK, st, &g_prof);
  cudaError_t e2 = cudaFreeAsync(d, st);
  if (e != cudaSuccess) return cuda_fail(e, "grouped launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "segment table free");
  return GL_OK;
}

const char* gl_error_string(int code) {
  switch (code) {
    case GL_OK: return "GL_OK";
    case GL_ERR_INVALID_ARG: return "GL_ERR_INVALID_ARG";
    case GL_ERR_OOM: return "GL_ERR_OOM";
    case GL_ERR_CUDA: return "GL_ERR_CUDA";
    case GL_ERR_TIMEOUT: return "GL_ERR_TIMEOUT";
    case GL_ERR_BUDGET: return "GL_ERR_BUDGET";
    case GL_ERR_UNSUPPORTED: return "GL_ERR_UNSUPPORTED";
    default: return "GL_ERR_UNKNOWN";
  }
}

const char* gl_last_error_message(void) { return g_msg; }

int gl_profile_enable(int on) {
  g_prof.drain();
  g_prof.on = on != 0;
  return GL_OK;
}

int gl_profile_select(unsigned kinds) {
  g_prof.drain();
  g_prof.kinds = kinds;
  return GL_OK;
}

int gl_profile_reset(void) {
  g_prof.drain();
  for (int i = 0; i < GL_KERNEL_KINDS; ++i) {
    g_prof.launches[i] = 0;
    g_prof.ms[i] = 0.0;
  }
  return GL_OK;
}

int gl_profile_read(long long* launches, double* total_ms) {
  g_prof.drain();
  for (int i = 0; i < GL_KERNEL_KINDS; ++i) {
    if (launches) launches[i] = g_prof.launches[i];
    if (total_ms) total_ms[i] = g_prof.ms[i];
  }
  return GL_OK;
}

const char* gl_kernel_name(int kind) {
  static const char* names[GL_KERNEL_KINDS] = {"k_setup", "k_ray_fwd", "k_conv", "k_ray_adj", "k_final", "other",
                                                   "k_order"};
  return (kind >= 0 && kind < GL_KERNEL_KINDS) ? names[kind] : "unknown";
}

long long gl_launch_count(void) { return g_launches.load(); }

}  // extern "C"
