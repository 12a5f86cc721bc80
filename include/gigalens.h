/*
 * gigalens.h - C ABI of the GB300 (sm_103a) batched lens-model likelihood.
 *
 * The library evaluates, for B parameter vectors of one lens system at a time
 * (or of several systems in one grouped launch), the forward model of
 * GIGA-Lens (arXiv:2202.07663, Sec. 2.1.1), its Gaussian log-likelihood with
 * model-dependent variance (Sec. 2.1.2, Eq. model-def) and the gradient of
 * that log-likelihood with respect to the 22 physical parameters (Sec. 2.2).
 *
 * Conventions shared by every entry point:
 *  - Parameter vectors are rows of GL_NPARAM = 22 float32 values in the order
 *    of Table 2: thetaE, gamma_epl, e_epl1, e_epl2, x_epl, y_epl, gamma_ext1,
 *    gamma_ext2, R_l, n_l, e_l1, e_l2, x_l, y_l, I_l, R_s, n_s, e_s1, e_s2,
 *    x_s, y_s, I_s. Positions and radii in arcsec, amplitudes in counts/s.
 *  - Images are row-major float32 [H, W]; row i has y = (i - (H-1)/2) * pixel
 *    scale and column j has x = (j - (W-1)/2) * pixel scale (pixel centres
 *    symmetric about the origin). The k-times supersampled grid follows the
 *    same rule at pixel scale / k (Sec. 2.1.1, last paragraph).
 *  - Unless a name ends in _host, every pointer argument other than the
 *    gl_system handle is DEVICE memory owned by the caller, and every call is
 *    asynchronous on the given CUDA stream (cudaStream_t passed as void*;
 *    NULL means the legacy default stream). Results are valid once the
 *    stream has reached the call.
 *  - Every call returns GL_OK (0) or a negative GL_ERR_* code; no exception
 *    or abort crosses the ABI. gl_error_string() names a code and
 *    gl_last_error_message() gives detail for the calling thread.
 *  - A vector with a non-finite entry, or |e| >= 1 for any of the three
 *    ellipticities, or R <= 0 or n <= 0 for a light profile, is not an error:
 *    its log-likelihood, chi^2 and gradient come back as NaN.
 *  - Calls on one gl_system share its scratch memory: issue them on one
 *    stream (or serialise them). Different systems are independent.
 *  - A gl_system lives on the device that was current when it was created.
 *    Every call that takes one must be made with that device current (the
 *    stream and the buffers belong to it too); otherwise the call returns
 *    GL_ERR_INVALID_ARG before anything is launched. The library never
 *    switches the current device for a call, except that gl_system_destroy
 *    frees on the system's own device and then restores the caller's.
 */
#ifndef GIGALENS_H_
#define GIGALENS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GL_NPARAM 22

enum gl_status {
  GL_OK = 0,
  GL_ERR_INVALID_ARG = -1, /* bad pointer, size or value; nothing was launched */
  GL_ERR_OOM = -2,         /* device or pinned allocation failed */
  GL_ERR_CUDA = -3,        /* a CUDA runtime call failed; see gl_last_error_message */
  GL_ERR_TIMEOUT = -4,     /* reserved: no call returns it (no kernel of the library waits on a flag) */
  GL_ERR_BUDGET = -5,      /* request exceeds the caller's memory budget */
  GL_ERR_UNSUPPORTED = -6  /* shape outside what the kernels support (e.g. image too large) */
};

typedef struct gl_system gl_system;

/*
 * gl_system_create - upload one lens system and keep it resident.
 *
 * Defines the data of the likelihood of Sec. 2.1.2 (Eq. model-def): the
 * observed image I_obs (counts/s), the background noise sigma_bkg, the PSF
 * and the exposure term G * t_exp; and the pixel grid of Sec. 2.1.1
 * (detector pixel scale, supersampling factor k_super).
 *
 *  out           receives the handle (host pointer to a gl_system*).
 *  image         HOST float32 [H, W], observed image I_obs.
 *  noise_map     HOST float32 [H, W], per-pixel background standard
 *                deviation sigma_bkg (> 0), or NULL with sigma_bkg_scalar.
 *  sigma_bkg     used for every pixel when noise_map is NULL (> 0).
 *  H, W          image size, 1 <= H, W <= 4096.
 *  psf           HOST float32 [K, K], used as given (not renormalised).
 *  K             PSF side, odd, 1 <= K <= 63.
 *  pixel_scale   arcsec per detector pixel (> 0). The Sersic amplitudes are
 *                surface brightness (counts/s/arcsec^2); a model pixel holds
 *                the flux falling on it, the mean over its k x k subpixels
 *                times pixel_scale^2 (counts/s), before the PSF.
 *  supersample   k_super >= 1 (<= 16).
 *  gain_exposure G * t_exp in seconds; <= 0 drops the Poisson term of the
 *                variance (sigma_tot^2 = sigma_bkg^2).
 *  stream        stream for the uploads; the call returns after they finish.
 *
 * The library copies every input; the caller keeps its buffers. Errors:
 * GL_ERR_INVALID_ARG for bad sizes, pointers or values; GL_ERR_UNSUPPORTED
 * when the zero-padded image does not fit the shared-memory convolution
 * stage (PSF sides 11 and 21: (H + K - 1) * P * 4 bytes + 2 K round4(K) * 4,
 * P = ceil(W/16)*16 + K - 1 rounded up to a multiple of 4 with an odd number
 * of 16-byte words; other sides: (ceil(H/8)*8 + K - 1) * (W + K - 1) * 4 +
 * 2 round4(K*K) * 4; either must stay below 220 KiB); GL_ERR_OOM /
 * GL_ERR_CUDA on device failures.
 */
int gl_system_create(gl_system** out, const float* image, const float* noise_map, float sigma_bkg,
                     int H, int W, const float* psf, int K, double pixel_scale, int supersample,
                     double gain_exposure, void* stream);

/*
 * gl_system_create_obsvar - the same system with the variance map built from
 *   the observed image, the alternative of Sec. 2.1.2:
 *   sigma_tot^2 = sigma_bkg^2 + max(I_obs, 0) / (G t_exp) per pixel (negative
 *   observed pixels count as zero), fixed at creation; the model-dependent
 *   Poisson term is off (gain_exposure only enters the map). Arguments and
 *   errors as gl_system_create.
 */
int gl_system_create_obsvar(gl_system** out, const float* image, const float* noise_map, float sigma_bkg,
                            int H, int W, const float* psf, int K, double pixel_scale, int supersample,
                            double gain_exposure, void* stream);

/*
 * gl_psf_factor - the PSF as a sum of separable terms (host only; touches no
 *   device). The convolution of Eq. 4's model (and its adjoint) with a PSF
 *   P = sum_{r<R} u_r v_r^T is R pairs of 1-D passes, 2 K R multiply-adds per
 *   pixel instead of K^2. gl_system_create applies this to its PSF: when
 *   R > 0 and the PSF side is 11 or 21 it keeps the factors
 *   (gl_system_psf_rank) and convolves that way, the whole image in one
 *   block when its R + 1 padded buffers fit 200 KiB of shared memory
 *   ((R + 1) * (ceil(H/8)*8 + K - 1) * P * 4 bytes, P as below), else (and
 *   for batches below half as many vectors as SMs) in row bands over a
 *   thread-block cluster. Grouped and batched calls use the factors where
 *   the whole image fits and the K x K stencil otherwise. A sampled
 *   Gaussian PSF has R = 1. The oracle's 2-D convolution is the reference
 *   for every form.
 *  psf    [K][K] row-major floats (the PSF as the system stores it).
 *  K      odd side, 1..255.
 *  fac    NULL, or room for fac_len floats: on return [R][2][K], the row
 *         factor sigma_r u_r then the column factor v_r of term r, from a
 *         singular value decomposition in FP64 (one-sided Jacobi).
 *  rank   out: R, the fewest terms whose dropped singular values have a root
 *         sum of squares of at most 2^-24 ||P||_F (the rounding the FP32
 *         entries already carry), or 0 when 4 R > K (the 2-D convolution is
 *         kept).
 * Errors: GL_ERR_INVALID_ARG for null psf/rank, a bad K, a non-finite value,
 * or fac_len < 2 R K with fac non-NULL.
 */
int gl_psf_factor(const float* psf, int K, float* fac, int fac_len, int* rank);

/* The number of separable PSF terms the system's single calls convolve
 * with (0: the K x K stencil), or GL_ERR_INVALID_ARG for NULL. Host state
 * only. */
int gl_system_psf_rank(const gl_system* sys);

/* Free the system, its resident data and its scratch. Synchronises the
 * device first. NULL is accepted. */
int gl_system_destroy(gl_system* sys);

/* Pre-size the system's scratch for batches of up to B vectors so that later
 * calls with B' <= B allocate nothing. */
int gl_system_reserve(gl_system* sys, int B);

/* Device bytes the system's scratch needs for a batch of B vectors. */
size_t gl_system_scratch_bytes(const gl_system* sys, int B);

/* Device bytes held by the resident data (image, variance, PSF and its
 * separable terms). */
size_t gl_system_resident_bytes(const gl_system* sys);

/* Device bytes of scratch (per-vector constants, image work buffer, tile
 * partials) the system holds now: 0 after creation, grown by calls that
 * need more and by gl_system_reserve; gl_loglik_grad_noalloc never grows it.
 * NULL gives 0. */
size_t gl_system_scratch_held(const gl_system* sys);

/*
 * gl_loglik - log-likelihood of B parameter vectors (Sec. 2.1.2, Eq.
 * model-def):
 *   log L = -1/2 sum_pixels [ (I_obs - I_model)^2 / s2 + ln(2 pi s2) ],
 *   s2 = sigma_bkg^2 + I_model / (G t_exp),
 * with I_model the PSF-convolved, k x k averaged, supersampled image of
 * Sec. 2.1.1. Arithmetic is float32 per ray and per pixel; each vector's sum
 * is accumulated in float64.
 *
 *  params      device float32 [B, 22].
 *  B           number of vectors, 0 <= B <= 2^24 (B = 0 does nothing).
 *  loglik_out  device float64 [B].
 *  chi2_out    device float64 [B] (first term of the sum, Sec. 2.1.2
 *              Eq. chi^2), or NULL.
 */
int gl_loglik(gl_system* sys, const float* params, int B, double* loglik_out, double* chi2_out, void* stream);

/*
 * gl_loglik_grad - gl_loglik plus d log L / d params (Sec. 2.2), computed
 * by a hand-written adjoint: the pixel adjoint is correlated with the PSF
 * and spread over the k x k subpixels, then every ray is recomputed and its
 * forward-mode derivatives are contracted with that adjoint. No ray position
 * is stored.
 *
 *  grad_out    device float64 [B, 22], same order as params.
 */
int gl_loglik_grad(gl_system* sys, const float* params, int B, double* loglik_out, double* chi2_out,
                   double* grad_out, void* stream);

/*
 * gl_loglik_grad_host - gl_loglik_grad with HOST buffers: copies params in,
 * computes, copies the results out and synchronises the stream before
 * returning. params/loglik_out/grad_out are host memory (pinned is fastest);
 * chi2_out may be NULL.
 */
int gl_loglik_grad_host(gl_system* sys, const float* params, int B, double* loglik_out, double* chi2_out,
                        double* grad_out, void* stream);

/*
 * gl_simulate - noiseless model images I_model (Sec. 2.1.1): ray-shoot the
 * supersampled grid, add lens light, average k x k, convolve with the PSF.
 *
 *  images_out  device float32 [B, H, W].
 */
int gl_simulate(gl_system* sys, const float* params, int B, float* images_out, void* stream);

/*
 * Grouped launch over several systems (continuous batching): one set of
 * kernel launches covers n (system, batch) segments. For segment s,
 * params[s] is device float32 [B[s], 22], loglik_out[s] device float64
 * [B[s]] and grad_out[s] device float64 [B[s], 22] or NULL (log L only).
 * chi2_out may be NULL or hold NULL entries. The host arrays are read before
 * the call returns. A system may appear in at most one segment of a call.
 * 1 <= n <= GL_MAX_SEGMENTS.
 */
#define GL_MAX_SEGMENTS 256
int gl_loglik_grad_grouped(gl_system* const* systems, const float* const* params, const int* B,
                           double* const* loglik_out, double* const* chi2_out, double* const* grad_out, int n,
                           void* stream);

/*
 * gl_loglik_grad_noalloc - gl_loglik_grad for callers that cannot allocate
 * device memory while they evaluate the likelihood: code running inside an
 * allocator or memory-pool callback, processes whose device memory is
 * entirely held by another framework's caching allocator, and hosts that
 * forbid allocation after start-up. The paper has no counterpart; it is a
 * deployment variant of the same computation.
 *
 * Arguments, results and errors are those of gl_loglik_grad. The call
 * allocates nothing: the kernels' scratch (per-vector constants, image work
 * buffer, per-tile gradient partials) lives in one static device array of
 * 32 MiB (33,554,432 bytes), which every GPU that loads
 * the library holds until the process exits. A batch whose scratch does not
 * fit is rejected with GL_ERR_INVALID_ARG before anything is launched (about
 * 2,100 vectors of a 60 x 60 image; scratch per vector is 4*H*W + 1,232
 * bytes plus 192 bytes per ray tile, gl_system_scratch_bytes(sys, B) / B).
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress)
 * with the system's device current; the lookup allocates nothing. The first
 * call on a device may also load the library's device code there, so make
 * it before any stream capture. Every call shares the one array and leaves
 * its contents behind; nothing in it has to start at zero. Calls whose
 * kernels overlap on the GPU (two streams, or two host threads) race on the
 * array: issue them on one stream.
 */
int gl_loglik_grad_noalloc(gl_system* sys, const float* params, int B, double* loglik_out, double* chi2_out,
                           double* grad_out, void* stream);

/*
 * Continuous batching (serving). A gl_batcher evaluates log-likelihood and
 * gradient for up to max_segments (system, vector range) segments in one
 * replay of a CUDA graph captured at creation. The graph's kernels use
 * persistent grids and read the batch composition from a device-resident
 * table, so every batch composition replays the same graph. The batcher owns
 * the scratch of a batch: arena_bytes of device memory shared by all its
 * segments (gl_batcher_segment_bytes gives one segment's share), so memory
 * scales with the vectors in flight, not with the number of resident systems.
 *
 * gl_batcher_create - allocates the arena, the device table and two pinned
 *   staging buffers, and captures the graph. Images up to max_H x max_W and
 *   PSFs up to max_K (odd) are accepted later. Errors: GL_ERR_INVALID_ARG,
 *   GL_ERR_UNSUPPORTED (max image too large for the shared-memory
 *   convolution), GL_ERR_OOM, GL_ERR_CUDA.
 *
 * gl_batcher_run - one batch: for segment s, params[s] device float32
 *   [B[s], 22], loglik_out[s] device float64 [B[s]], grad_out[s] device
 *   float64 [B[s], 22], chi2_out NULL or per segment NULL / [B[s]]. A system
 *   may appear in several segments. Host arrays are read before return; the
 *   work is asynchronous on stream. Runs of one batcher share its arena and
 *   device table, so they execute one after another: a run issued on another
 *   stream than the previous run's first waits (on the device) for that run
 *   to finish. Make the calls from one host thread at a time. A batch of one
 *   non-empty segment runs the launch sequence of a single-system call
 *   (gl_loglik_grad's, with its share of the arena as scratch) instead of the
 *   graph, so its results are those of gl_loglik_grad, bit for bit. The call blocks
 *   only if the staging buffer it reuses is still being copied (two batches
 *   back). Errors: GL_ERR_BUDGET if the segments' scratch exceeds the arena,
 *   GL_ERR_UNSUPPORTED for a segment beyond max_H/max_W/max_K.
 */
typedef struct gl_batcher gl_batcher;
int gl_batcher_create(gl_batcher** out, int max_segments, size_t arena_bytes, int max_H, int max_W, int max_K);
int gl_batcher_destroy(gl_batcher* b);
size_t gl_batcher_segment_bytes(const gl_system* sys, int B);
int gl_batcher_run(gl_batcher* b, gl_system* const* systems, const float* const* params, const int* B,
                   double* const* loglik_out, double* const* chi2_out, double* const* grad_out, int n, void* stream);

/*
 * Multi-start MAP (Sec. 2.3) in the unconstrained parameters of Sec. 2.2.
 *
 * gl_prior_entry describes one parameter's prior marginal (Eq. sim-dist):
 *   GL_PRIOR_NORMAL       a = mean, b = standard deviation
 *   GL_PRIOR_LOGNORMAL    a = median, b = standard deviation of the log
 *   GL_PRIOR_TRUNCNORMAL  a = mean, b = standard deviation, [c, d] = support
 *   GL_PRIOR_UNIFORM      [a, b] = support
 * The bijector g (Sec. 2.2, Eq. exp, Eq. sigmoid) follows the support:
 * exp for log-normal, a + (b - a) sigmoid(z) for truncated-normal and
 * uniform, identity for normal. prior points to GL_NPARAM host entries.
 *
 * gl_map_inverse   - z = g^-1(theta) for theta device float32 [B, 22]
 *                    (start points drawn in physical parameters).
 * gl_map_transform - theta = g(z) as float32, for the likelihood call.
 * gl_map_adam_step - given log L and d log L / d theta at theta = g(z)
 *   (device float64 [B], [B, 22]), computes the objective
 *   f(z) = -(log L + log p(g(z)) + log|J|) of Eq. obj-fun into
 *   objective_out (may be NULL), its gradient in z, the Adam update
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   z -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 *   with step count t >= 1 (skipped when m and v are NULL), and writes
 *   theta_out = g(z) after the update (may be NULL). State z, m, v is device
 *   float64 [B, 22]. FP64 arithmetic, one warp per start.
 */
#define GL_PRIOR_NORMAL 0
#define GL_PRIOR_LOGNORMAL 1
#define GL_PRIOR_TRUNCNORMAL 2
#define GL_PRIOR_UNIFORM 3
typedef struct gl_prior_entry {
  int kind;
  int reserved;
  double a, b, c, d;
} gl_prior_entry;
int gl_map_inverse(int B, const float* theta, const gl_prior_entry* prior, double* z_out, void* stream);
int gl_map_transform(int B, const double* z, const gl_prior_entry* prior, float* theta_out, void* stream);
int gl_map_adam_step(int B, double* z, double* m, double* v, int t, double lr, double beta1, double beta2, double eps,
                     const double* loglik, const double* grad_theta, const gl_prior_entry* prior,
                     double* objective_out, float* theta_out, void* stream);

/*
 * gl_posterior_grad - the log density of the unconstrained parameters,
 *   log p~(z) = log L + log p(g(z)) + log|J| (Eq. reparam-post; the
 *   negative of the MAP objective), and its gradient in z, given log L and
 *   d log L / d theta at theta = g(z). logp_out device float64 [B],
 *   grad_z_out device float64 [B, 22]. grad_theta may be NULL (then
 *   grad_z_out is not written and may be NULL too): log density only. Used
 *   by HMC on the posterior and by VI.
 */
int gl_posterior_grad(int B, const double* z, const double* loglik, const double* grad_theta,
                      const gl_prior_entry* prior, double* logp_out, double* grad_z_out, void* stream);

/*
 * Hamiltonian Monte Carlo around the gradient (Sec. 2.5; Table 1 sampler
 * settings are the caller's). Chain state is FP64 on the device: positions
 * q [B, d], momenta p [B, d], log density logp [B], its gradient [B, d];
 * inv_mass [d] is the diagonal of the inverse mass matrix. The caller draws
 * the random numbers (initial momenta, log-uniforms for the accept test).
 *
 * gl_hmc_leapfrog - one leapfrog update: p += kick * eps * grad, then
 *   q += eps * inv_mass * p, and q32_out = (float)q for the next likelihood
 *   call (q32_out may be NULL when q is not the likelihood's input, e.g.
 *   unconstrained parameters). kick = 0.5 for the first step of a
 *   trajectory, 1 afterwards (the half kicks at both ends of consecutive
 *   steps merged).
 *
 * gl_hmc_finish - last half kick p += eps/2 * grad_new, Hamiltonians
 *   H = -logp + 1/2 sum p^2 inv_mass of the start (p0, logp0) and end
 *   (p, logp_new) points in FP64, accept where log_u < H_start - H_end (and
 *   both are finite); accepted chains copy q_new, logp_new, grad_new into q,
 *   logp, grad. accepted[b] is 1 or 0; accept_prob[b] (may be NULL) receives
 *   min(1, exp(H_start - H_end)), 0 for a non-finite Hamiltonian.
 *
 * All pointers are device memory; asynchronous on stream; 1 <= d <= 4096.
 */
int gl_hmc_leapfrog(int B, int d, double* q, double* p, const double* grad, const double* inv_mass, double eps,
                    double kick, float* q32_out, void* stream);
/* gl_hmc_leapfrog_dev - gl_hmc_leapfrog with eps read from device memory
 *   (eps_dev, one float64) when the kernel runs, so that a captured CUDA
 *   graph of a leapfrog step can be replayed while the step size changes. */
int gl_hmc_leapfrog_dev(int B, int d, double* q, double* p, const double* grad, const double* inv_mass,
                        const double* eps_dev, double kick, float* q32_out, void* stream);
int gl_hmc_finish(int B, int d, const double* p0, const double* logp0, double* p, const double* grad_new,
                  const double* logp_new, const double* q_new, const double* inv_mass, const double* log_u,
                  double eps, double* q, double* logp, double* grad, int* accepted, double* accept_prob,
                  void* stream);

/*
 * gl_hmc_chees - the trajectory-length gradient of the ChEES criterion
 *   (Hoffman, Radul & Sountsov 2021), which Sec. 2.5 adapts during the first
 *   80% of burn-in. For chains b with start q_prev[b], proposal q_prop[b] and
 *   end momentum p_prop[b] after a trajectory of length t:
 *   a_b = |q_prop[b] - m'|^2 - |q_prev[b] - m|^2, c_b = (q_prop[b] - m') .
 *   (inv_mass * p_prop[b]), m and m' the chain means (m' over finite
 *   proposals); out[0] = sum w t a c / sum w (gradient in log T),
 *   out[1] = sum w a^2/4 / sum w (the criterion), out[2] = sum w, with
 *   w = accept_prob; chains with a non-finite proposal, momentum or weight
 *   are left out; sum w = 0 gives zeros. Device float64 arrays [B, d], [d],
 *   [B], out [3]; 1 <= B <= GL_HMC_CHEES_MAX_B, 1 <= d <= GL_HMC_CHEES_MAX_D.
 *   Fixed reduction order: equal inputs give equal outputs.
 */
#define GL_HMC_CHEES_MAX_B 16384
#define GL_HMC_CHEES_MAX_D 1024
int gl_hmc_chees(int B, int d, const double* q_prev, const double* q_prop, const double* p_prop,
                 const double* inv_mass, const double* accept_prob, double t, double* out, void* stream);

/*
 * The whitened posterior in two calls (the HMC preconditioning of Sec. 2.5 on
 * the posterior of the unconstrained parameters, Eq. reparam-post), one
 * warp per chain, d = 22:
 * gl_posterior_whitened_transform - z_out = mu + L x (L lower triangular,
 *   row-major 22 x 22 float64; the sums of gl_hmc_affine) and
 *   theta_out = (float) g(z) (the bijectors of gl_map_transform);
 * gl_posterior_whitened_grad - logp_out = loglik + log p(g(z)) + log|J| and,
 *   with grad_theta (d log L / d theta at theta), grad_x_out = L^T grad_z
 *   (gl_posterior_grad followed by gl_hmc_affine_pullback: the same sums).
 * Between them the caller evaluates log L and its gradient at theta_out.
 * Device pointers: x, z_out [B, 22] float64; theta_out [B, 22] float32;
 * loglik, logp_out [B]; grad_theta, grad_x_out [B, 22]; mu [22]. Outputs must
 * not alias inputs; GL_ERR_INVALID_ARG for a bad prior table, B < 0 or a
 * null pointer.
 */
int gl_posterior_whitened_transform(int B, const double* x, const double* mu, const double* L,
                                    const gl_prior_entry* prior, double* z_out, float* theta_out, void* stream);
int gl_posterior_whitened_grad(int B, const double* z, const double* loglik, const double* grad_theta,
                               const double* L, const gl_prior_entry* prior, double* logp_out, double* grad_x_out,
                               void* stream);
/*
 * gl_hmc_leapfrog_whitened - one leapfrog update of HMC on the whitened
 *   coordinates (identity mass on x would be inv_mass = 1): p += kick eps grad,
 *   x += eps inv_mass p (gl_hmc_leapfrog's arithmetic; eps from *eps_dev when
 *   eps_dev is not NULL), then gl_posterior_whitened_transform at the new x,
 *   in one launch. x, p, grad [B, 22] float64 (x and p updated in place),
 *   inv_mass [22]; other arguments as for gl_posterior_whitened_transform.
 */
int gl_hmc_leapfrog_whitened(int B, double* x, double* p, const double* grad, const double* inv_mass, double eps,
                             const double* eps_dev, double kick, const double* mu, const double* L,
                             const gl_prior_entry* prior, double* z_out, float* theta_out, void* stream);
/*
 * gl_hmc_leapfrog_whitened_chain - a leapfrog step after the first of a
 *   trajectory, in one launch: the whitened posterior's gradient at the
 *   current point (grad_x of gl_posterior_whitened_grad, same sums; its log p~
 *   is not formed), then gl_hmc_leapfrog_whitened with that gradient.
 *   z [B, 22] float64 is read as the current point (the z_out of the previous
 *   step) and overwritten with the new one; grad_theta [B, 22] is
 *   d log L / d theta at the current point's theta. x, p, inv_mass, eps,
 *   eps_dev, kick, mu, L, prior, theta_out as for gl_hmc_leapfrog_whitened.
 *   A trajectory of n steps is gl_hmc_leapfrog_whitened (kick 1/2), then n - 1
 *   of these (kick 1) with log L evaluated after each launch, then
 *   gl_posterior_whitened_grad at the last point: the bits of n pairs of
 *   gl_hmc_leapfrog_whitened and gl_posterior_whitened_grad.
 *   GL_ERR_INVALID_ARG for a bad prior table, B < 0, a null pointer, a
 *   non-finite eps (eps_dev NULL) or aliased x, p, z, grad_theta.
 */
int gl_hmc_leapfrog_whitened_chain(int B, double* x, double* p, double* z, const double* grad_theta,
                                   const double* inv_mass, double eps, const double* eps_dev, double kick,
                                   const double* mu, const double* L, const gl_prior_entry* prior, float* theta_out,
                                   void* stream);

/*
 * Dense preconditioning (Sec. 2.5: the mass matrix set to the inverse of a
 * posterior covariance Sigma = L L^T, e.g. the variational one). HMC with
 * identity mass on whitened coordinates x is HMC with mass Sigma^-1 on
 * z = mu + L x, so the sampler keeps its diagonal kernels and the target
 * maps through these two calls.
 *
 * gl_hmc_affine - z_out = mu + L x per chain; L lower triangular, row-major
 *   d x d float64 (entries above the diagonal are ignored); z32_out
 *   (may be NULL) receives (float)z. x [B, d], mu [d], z_out [B, d].
 * gl_hmc_affine_pullback - grad_x_out = L^T grad_z per chain.
 *
 * Device pointers; outputs must not alias inputs; 1 <= d <= GL_HMC_AFFINE_MAX_D.
 */
#define GL_HMC_AFFINE_MAX_D 64
int gl_hmc_affine(int B, int d, const double* x, const double* mu, const double* L, double* z_out, float* z32_out,
                  void* stream);
int gl_hmc_affine_pullback(int B, int d, const double* grad_z, const double* L, double* grad_x_out, void* stream);

/*
 * Full-rank variational inference (Sec. 2.4; Table 1 settings are the
 * caller's). The surrogate posterior over the unconstrained parameters is
 * q = N(mu, L L^T) with L from the Cholesky bijector: phi = [mu (d),
 * u (d(d+1)/2)], u packed row by row, u[i(i+1)/2 + j] = L[i][j] for j < i and
 * log L[i][i] for j = i. The caller draws eps ~ N(0, I) [n, d] and evaluates
 * log p~ (and its gradient in z for the pathwise estimator) at the draws.
 *
 * gl_vi_param_count - d + d(d+1)/2 (0 for d outside 1..GL_VI_MAX_D).
 * gl_vi_workspace_bytes - device scratch gl_vi_step needs for n draws.
 *
 * gl_vi_sample - z_out = mu + L eps per draw [n, d] float64; theta_out
 *   (may be NULL) receives g(z) as float32 through the prior's bijector
 *   when prior != NULL (then d must be GL_NPARAM), else (float)z.
 *
 * gl_vi_step - the ELBO loss estimate mean(log q(z_s) - log p~(z_s)) into
 *   loss_out [1] and its gradient in phi into grad_out [P] by
 *   GL_VI_SCORE: Eq. elbo-grad, mean((log q - log p~) d log q / d phi) with
 *     the draws held fixed (grad_z unused, may be NULL); or
 *   GL_VI_PATHWISE: the reparameterised gradient through z = mu + L eps
 *     (grad_z [n, d] = d log p~ / dz required).
 *   With m and v (both [P]) given, one Adam step t >= 1 updates phi in place:
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   phi -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + adam_eps); with both
 *   NULL phi is left alone. workspace: gl_vi_workspace_bytes(n, d) bytes of
 *   device memory owned by the caller. Sums run in a fixed order: equal
 *   inputs give equal outputs. logp, eps, grad_z, phi, m, v, grad_out,
 *   loss_out are device float64; asynchronous on stream.
 */
#define GL_VI_MAX_D 32
#define GL_VI_SCORE 0
#define GL_VI_PATHWISE 1
size_t gl_vi_param_count(int d);
size_t gl_vi_workspace_bytes(int n, int d);
int gl_vi_sample(int n, int d, const double* eps, const double* phi, const gl_prior_entry* prior, double* z_out,
                 float* theta_out, void* stream);
int gl_vi_step(int n, int d, const double* eps, const double* logp, const double* grad_z, int estimator,
               double* phi, double* m, double* v, int t, double lr, double beta1, double beta2, double adam_eps,
               double* grad_out, double* loss_out, void* workspace, void* stream);

/*
 * The two halves of gl_vi_step, for draws spread over several processes:
 * gl_vi_moments - the estimator's moment sums over this call's n draws
 *   (sums_out: device float64 [1 + gl_vi_param_count(d)], not divided by n);
 *   the caller gathers the processes' sums, one row each, and passes them to
 * gl_vi_apply - the loss, gradient and (with m, v) Adam step from sums
 *   [nparts, 1 + gl_vi_param_count(d)] over n_total draws in all; the rows are
 *   added in row order, so every process that passes the same rows gets the
 *   same bits. Other arguments mean what they mean for gl_vi_step.
 * One process: gl_vi_moments then gl_vi_apply(n, d, 1, ...) gives gl_vi_step's
 * bits. Errors: GL_ERR_INVALID_ARG for a size out of range or a null pointer.
 */
int gl_vi_moments(int n, int d, const double* eps, const double* logp, const double* grad_z, int estimator,
                  const double* phi, void* workspace, double* sums_out, void* stream);
int gl_vi_apply(int n_total, int d, int nparts, const double* sums, int estimator, double* phi, double* m, double* v, int t,
                double lr, double beta1, double beta2, double adam_eps, double* grad_out, double* loss_out,
                void* stream);

/*
 * gl_loglik_grad_profiled - log L profiled over the two light amplitudes
 *   (Sec. 2.1.2: with a parameter-independent variance the model is linear in
 *   I_l and I_s, so they are solved in closed form). Per vector: the model
 *   images A_l, A_s at unit amplitudes, the 2x2 weighted least-squares solve
 *   [<A_l,A_l> <A_l,A_s>; <A_s,A_l> <A_s,A_s>] [I_l; I_s] = [<A_l,D>; <A_s,D>]
 *   (<a,b> = sum a b / sigma_tot^2; FP64), then log L and chi^2 of
 *   M = I_l A_l + I_s A_s (the PSF convolution is linear, so the convolved
 *   basis images give the convolved model; no second forward pass) and the
 *   gradient at the solved amplitudes from d log L / d M by the PSF
 *   correlation and the ray adjoint. Where the system is singular (a self-product
 *   below 1e-12 of the other, or det below 1e-12 of the diagonal product) the
 *   amplitude with the smaller self-product is 0 and the other is solved
 *   alone. The input's I_l and I_s are ignored; grad_out entries 14 and 21
 *   are 0 (the profiled log L does not depend on them) and the other 20 are
 *   the profiled gradient. amps_out (may be NULL) receives [B, 2] float64
 *   (I_l, I_s); chi2_out and grad_out may be NULL. Needs a system whose
 *   variance does not depend on the model (gl_system_create_obsvar, or
 *   gain_exposure <= 0), else GL_ERR_INVALID_ARG; 0 <= B <= 2^23. Device
 *   pointers; asynchronous on stream; scratch for 2B basis images is held by
 *   the system and grows on demand.
 */
int gl_loglik_grad_profiled(gl_system* sys, const float* params, int B, double* loglik_out, double* chi2_out,
                            double* grad_out, double* amps_out, void* stream);

/* Name of a status code (static string). */
const char* gl_error_string(int code);

/* Detail of the calling thread's last error (static per-thread buffer). */
const char* gl_last_error_message(void);

/*
 * Instrumentation. When enabled, every kernel the library launches of the
 * selected kinds (gl_profile_select: bit k for kind k; all kinds until
 * called) is bracketed by CUDA events recorded on the launching stream.
 * An event between two kernels of a call also ends their programmatic
 * overlap (the next kernel is launched only when the previous one has
 * finished), so bracketing every kernel lengthens a call; bracketing one
 * kind costs only its two boundaries. gl_profile_read synchronises on the
 * events and fills, per kernel kind (indices below), the number of launches
 * and the summed device time in milliseconds; arrays hold GL_KERNEL_KINDS
 * entries. gl_launch_count counts every kernel launch since load
 * (profiling on or off).
 */
#define GL_KERNEL_KINDS 7
enum gl_kernel_kind {
  GL_K_SETUP = 0,    /* per-vector constants */
  GL_K_RAY_FWD = 1,  /* ray shooting + lights + k x k binning */
  GL_K_CONV = 2,     /* PSF convolution + likelihood (+ pixel adjoint) */
  GL_K_RAY_ADJ = 3,  /* recomputed rays + forward-mode derivatives */
  GL_K_FINAL = 4,    /* per-vector gradient reduction */
  GL_K_OTHER = 5,
  GL_K_ORDER = 6     /* order of a call's vectors, longest EPL series first:
                        two kernels (keys, counting sort) in single-system
                        calls of at least one vector per SM */
};
int gl_profile_enable(int on);
int gl_profile_select(unsigned kinds);
int gl_profile_reset(void);
int gl_profile_read(long long* launches, double* total_ms);
const char* gl_kernel_name(int kind);
long long gl_launch_count(void);

/*
 * gl_profile_peak - measured throughput of one pipe of the current device,
 * the denominator of the likelihood kernels' roofline (they are bound by
 * FP32 arithmetic and the special-function unit, not by memory):
 *   GL_PEAK_FP32_FMA  FP32 flop/s of packed fused multiply-adds (FMA = 2 flops)
 *   GL_PEAK_MUFU_EX2  ex2.approx results/s of the special-function unit
 * Each is the best of five timed launches of a kernel of independent
 * dependency chains over every SM, at the clock the GPU runs at. rate_out is
 * a HOST double. Blocking (synchronises the launches on the legacy default
 * stream); allocates and frees a small device buffer. Errors:
 * GL_ERR_INVALID_ARG for a NULL rate_out or an unknown kind; GL_ERR_CUDA.
 */
#define GL_PEAK_FP32_FMA 0
#define GL_PEAK_MUFU_EX2 1
int gl_profile_peak(int kind, double* rate_out);

#ifdef __cplusplus
}
#endif

#endif /* GIGALENS_H_ */
