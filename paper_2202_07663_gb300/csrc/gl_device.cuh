// gl_device.cuh - device data layout and per-ray arithmetic of the lens model.
//
// Model (arXiv:2202.07663, Sec. 2.1.1): an elliptical power-law (EPL) mass
// plus external shear deflects each ray of a k-times supersampled pixel grid;
// the source Sersic is evaluated at the ray's source-plane position, the lens
// Sersic at its image-plane position; k x k rays are averaged to a detector
// pixel; the result is convolved with the PSF.
//
// The EPL is evaluated in a form derived for this code rather than in the
// paper's (q, phi, rotate, series, rotate back) sequence. With the complex
// ellipticity eps = e1 + i e2 = f e^{2 i phi}, f = (1-q)/(1+q), and the
// offset z = (x - x_c) + i (y - y_c) of a ray from the lens centre:
//
//   w   = z - eps conj(z)                 (= 2/(1+q) e^{i phi} (q x_l + i y_l))
//   rho^2 = |w|^2 / (1 - |eps|^2)         (= q x_l^2 + y_l^2 / q, the paper's
//                                          elliptical radius of Eq. kappa)
//   u   = -conj(eps) w / conj(w)          (= -f e^{2 i phi_ell}, Tessore & Metcalf)
//   F(u) = sum_n a_n u^n,  a_0 = 1,  a_n = a_{n-1} c_n,
//          c_n = (2n - 2 + t) / (2n + 2 - t),  t = gamma - 1
//        = 1 + u G(u),  G(u) = sum_{n>=0} a_{n+1} u^n
//   alpha = (thetaE / rho)^t  w  F(u)     (image frame, complex)
//
// This is the Tessore & Metcalf (2015) deflection that the paper cites,
// rotated back to the image frame, after the identities
//   2b/(1+q) (b/R)^(t-1) e^{i phi} e^{i phi_ell} = (thetaE/rho)^t w
// (b = thetaE sqrt(q), R = sqrt(q) rho) have been applied. It is smooth in
// (e1, e2) through e = 0, needs no atan2 and no rotation, and gives the
// gradient with respect to e1, e2 in closed form. G is evaluated by Horner's
// rule on the coefficients a_1..a_N (per-vector term count N, so all rays of
// a vector run the same loop): one complex multiply-add per term.
//
// The Sersic profile (Eq. Sersic) uses the same quadratic form for its
// elliptical radius: q x_l^2 + y_l^2 / q = A dx^2 + 2 B dx dy + C dy^2 with
// A = (1 + e^2 - 2 e1)/(1 - e^2), B = -2 e2/(1 - e^2), C = (1 + e^2 + 2 e1)/(1 - e^2),
// and is evaluated as I = I0 exp2(k1 (1 - s)), s = exp2(c1 log2(rho^2 / R_eff^2)),
// with c1 = 1/(2n), k1 = b_n / ln 2, b_n = 1.9992 n - 0.3271. The 1/R_eff^2 is
// folded into A, B, C, so log2 s has no cancelling offset.
//
// FP32 accuracy. The likelihood of a sharp, high signal-to-noise image is so
// steep in the parameters that an error which acts like a small parameter
// change (the same for every ray) moves the gradient by the Hessian times
// that change; rounding errors that differ from ray to ray mostly cancel in
// the pixel sums. So everything that is the same for all rays of a vector is
// formed in FP64 and rounded once: the ray grid (x = n h with n an integer
// and h = pixel_scale / (2k) as a pair of floats, instead of x0 + j sub with
// both constants rounded, which shifted the whole grid by ~1e-7 arcsec),
// log2(thetaE sqrt(1 - |eps|^2)) as a pair of floats, and the Sersic
// coefficients with 1/R_eff^2 folded in.
#pragma once

#include <cstdint>

namespace gl {

constexpr int NPARAM = 22;
constexpr int NMAX = 128;            // cap on EPL series terms per vector (a multiple of 32)
constexpr int NACC = 24;             // adjoint accumulators per vector
constexpr float RHO2_MIN = 1e-12f;   // (1e-6 arcsec)^2: EPL deflection zero / Sersic radius floor
constexpr int RAY_THREADS = 256;     // block size of the ray kernels
constexpr int FINAL_THREADS = 128;   // block size of k_final (vectors per block)

// Accumulator slots of the adjoint (per vector, before the chain rule).
enum Acc {
  A_THETAE = 0, A_T, A_E1, A_E2, A_XC, A_YC, A_G1, A_G2,            // mass (x b_s/n_s)
  A_L_R, A_L_N1, A_L_N2, A_L_E1, A_L_E2, A_L_X, A_L_Y, A_L_I,        // lens light
  A_S_R, A_S_N1, A_S_N2, A_S_E1, A_S_E2, A_S_X, A_S_Y, A_S_I         // source
};

struct LightC {
  float A, B2, C;          // rho^2 / R_eff^2 = A dx^2 + B2 dx dy + C dy^2 (B2 = 2B)
  float x, y;              // centre
  float c1;                // log2 s = c1 log2(rho^2 / R_eff^2)
  float r2min;             // RHO2_MIN / R_eff^2: floor of rho^2 / R_eff^2
  float k1;                // b_n / ln 2
  float I0;                // amplitude
  float A1, B21, C1;       // d(A, B2, C)/d e1
  float A2, B22, C2;       // d(A, B2, C)/d e2
};

struct __align__(16) VecConst {
  float xc, yc;            // EPL centre
  float e1, e2;            // EPL complex ellipticity
  float lc;                // log2(thetaE sqrt(1 - |eps|^2)) rounded: log2(thetaE / rho) = lc - log2(|w|^2) / 2
  float tlc_lo;            // t x (the rounding error of lc)
  float t;                 // gamma - 1
  float w2min;             // RHO2_MIN (1 - |eps|^2): |w|^2 below it is rho < 1e-6 arcsec
  float g1, g2;            // external shear
  int nterms;              // series terms of F (0 <= N <= NMAX); < 0 marks an invalid vector
  int nterms_adj;          // series terms in the adjoint, max(N, 1)
  float th;                // t / 2
  float kc;                // 1 - t/2, for dF/du = [(t/2) F - (1 - t/2) G] / (1 - u)
  float kap_c;             // (2 - t) / 2: kappa = kap_c (thetaE/rho)^t
  float omt;               // 1 - t
  float e1i, e2i;          // e1, e2 times 1 / (1 - |eps|^2)
  int order;               // written by k_order into slot p: the vector the ray kernels take p-th
  float pad_[3];
  LightC light[2];         // [0] lens light at theta, [1] source at beta
  float an[NMAX];          // a_n = c_1 ... c_n, n = 1..NMAX at index n-1
  float ant[NMAX];         // d a_n / d t
};
static_assert(sizeof(VecConst) % 16 == 0, "VecConst must be a whole number of 16-byte words");

// One (system, batch) segment of a launch.
struct Seg {
  // resident system
  const float* image;      // I_obs [H, W]
  const float* sigma2;     // sigma_bkg^2 [H, W]
  const float* psf;        // [K, K]
  const float* psf_sep;    // [psf_rank][2][K]: the PSF as separable terms (sigma_r u_r, v_r), or null
  int psf_rank;            // separable terms of the PSF (0: 2-D convolution only)
  int conv_sep;            // 1: this launch convolves with the separable terms (its shared memory has room)
  int H, W, K, k;
  float hh, hl;            // h = pixel_scale / (2k) = hh + hl (a pair of floats)
  int nx0, ny0;            // 1 - kW, 1 - kH: subpixel (i, j) sits at ((2j + nx0) h, (2i + ny0) h)
  float inv_gain;          // 1 / (G t_exp), 0 drops the Poisson term
  // this call
  const float* params;     // [B, 22]
  int B;
  int ntiles;              // ray tiles per vector
  int tile_pix;            // detector pixels per ray tile
  int ray_order;           // 1: the ray kernels take the vectors in VecConst::order (k_order); 0: as given
  double* loglik;          // [B] or null
  double* chi2;            // [B] or null
  double* grad;            // [B, 22] or null
  float* sim;              // [B, H, W] or null
  // scratch
  VecConst* vc;            // [B]
  float* work;             // [B, H, W]: binned pre-PSF image, then the subpixel adjoint
  double* partial;         // [B, ntiles, NACC]
  // first item of this segment in the launch's item spaces
  int vec_begin;           // per-vector kernels
  int ray_begin;           // ray kernels (B * ntiles items)
  int conv_begin;          // convolution kernel of this segment's PSF class
  int conv_two_buf;        // 1: pixel adjoint kept in a second shared-memory buffer
};

// Header of a device-resident segment table whose item counts the kernels
// read at run time (graph-replayed grouped launches).
constexpr int N_CONV_CLASSES = 3;
struct TableHdr {
  int nseg, vec_total, ray_total, pad_;
  int conv_first[N_CONV_CLASSES];
  int conv_nseg[N_CONV_CLASSES];
  int conv_total[N_CONV_CLASSES];
};

// ---------------------------------------------------------------- MUFU ----
// Single hardware instructions of the special-function unit.
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Coordinate n h of the supersampled grid (n = 2j + nx0, an odd or even
// integer) from h = hh + hl: the exact product n hh, the small n hl added
// before the one rounding, so a ray's position is off by at most about half
// an ulp of itself and the grid is neither shifted nor scaled.
__device__ __forceinline__ float grid_coord(int n, float hh, float hl) {
  const float f = float(n);
  return fmaf(f, hh, f * hl);
}

// ------------------------------------------- programmatic dependent launch ---
// The likelihood kernels of a call are launched with programmatic stream
// serialization. A kernel's blocks wait on the device for the previous grid
// to complete and its writes to be visible before they read anything (the
// constructor), and signal, when they are done, that the next grid may be
// scheduled (the destructor, on every exit path); the next grid is then
// launched while this one's last blocks drain. (Signalling at the start of
// a block instead let the next grid's blocks be placed on the SMs while this
// one still held them, and measured slower.) Without the launch attribute
// both instructions do nothing.
struct PdlScope {
  __device__ __forceinline__ PdlScope() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
  __device__ __forceinline__ ~PdlScope() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
};

// --------------------------------------------------------- packed pairs ---
// Two rays of one parameter vector evaluated in lockstep with Blackwell's
// packed FP32 instructions (one f32x2 FMA/MUL/ADD does the arithmetic of two
// rays in one issue slot). The ray kernels are issue-bound, so pairing rays
// halves the issue cost of their FP32 arithmetic. Special-function (MUFU)
// instructions and comparisons act on each half.
struct F2 {
  float2 v;
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ F2 operator-(F2 a) { return {__fmul2_rn(a.v, make_float2(-1.f, -1.f))}; }

template <class T> __device__ __forceinline__ T sp(float a);
template <> __device__ __forceinline__ float sp<float>(float a) { return a; }
template <> __device__ __forceinline__ F2 sp<F2>(float a) { return {make_float2(a, a)}; }

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ F2 fmaT(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ float ex2T(float a) { return ex2(a); }
__device__ __forceinline__ F2 ex2T(F2 a) { return {make_float2(ex2(a.v.x), ex2(a.v.y))}; }
__device__ __forceinline__ float lg2T(float a) { return lg2(a); }
__device__ __forceinline__ F2 lg2T(F2 a) { return {make_float2(lg2(a.v.x), lg2(a.v.y))}; }
__device__ __forceinline__ float rcpT(float a) { return rcp(a); }
__device__ __forceinline__ F2 rcpT(F2 a) { return {make_float2(rcp(a.v.x), rcp(a.v.y))}; }
__device__ __forceinline__ float maxT(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ F2 maxT(F2 a, F2 b) { return {make_float2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y))}; }
// 1 where a >= b, else 0
__device__ __forceinline__ float geT(float a, float b) { return a >= b ? 1.f : 0.f; }
__device__ __forceinline__ F2 geT(F2 a, F2 b) {
  return {make_float2(a.v.x >= b.v.x ? 1.f : 0.f, a.v.y >= b.v.y ? 1.f : 0.f)};
}

// log2 without the bias of lg2.approx. lg2.approx.ftz measured on GB300
// (2^26 arguments against FP64): error +6e-8 on average for x in [1/2, 2]
// and about +3e-8 |log2 x| elsewhere, always of one sign, which acts on the
// Sersic profile like a change of its parameters. One correction step: with
// y0 = lg2.approx(x), log2 x = y0 + log2(x 2^-y0) and x 2^-y0 - 1 (one FMA on
// ex2.approx(-y0), whose mean error is -8e-9) is ln 2 times that remainder
// to first order (the remainder is ~1e-7, its square negligible).
__device__ __forceinline__ float lg2c(float x) {
  const float y0 = lg2(x);
  const float d = fmaf(x, ex2(-y0), -1.f);
  return fmaf(d, 1.44269504088896341f, y0);
}
__device__ __forceinline__ float lg2cT(float a) { return lg2c(a); }
// The same correction on a packed pair: per lane the arithmetic of lg2c (the
// two FMAs as one packed FMA each).
__device__ __forceinline__ F2 lg2cT(F2 a) {
  const float y0x = lg2(a.v.x), y0y = lg2(a.v.y);
  const F2 e = {make_float2(ex2(-y0x), ex2(-y0y))};
  const F2 d = {__ffma2_rn(a.v, e.v, make_float2(-1.f, -1.f))};
  return {__ffma2_rn(d.v, make_float2(1.44269504088896341f, 1.44269504088896341f), make_float2(y0x, y0y))};
}

// The same for a packed pair of grid indices n already in float (exact: |n|
// is far below 2^24), so that the inner subpixel loops step n by exact float
// adds instead of converting an integer per ray.
__device__ __forceinline__ F2 grid_coord2(F2 n, float hh, float hl) { return fmaT(n, sp<F2>(hh), n * sp<F2>(hl)); }

// Elliptical Sersic at (px, py), generic in the ray type; the forward model,
// so its log2 is the unbiased one (log L sums the model over every pixel).
template <class T>
__device__ __forceinline__ T sersic_fwd_T(const LightC& L, T px, T py) {
  const T dx = px - sp<T>(L.x), dy = py - sp<T>(L.y);
  T r2 = fmaT(sp<T>(L.A) * dx, dx, fmaT(sp<T>(L.B2) * dx, dy, sp<T>(L.C) * dy * dy));
  r2 = maxT(r2, sp<T>(L.r2min));
  const T s = ex2T(sp<T>(L.c1) * lg2cT(r2));
  return sp<T>(L.I0) * ex2T(fmaT(sp<T>(-L.k1), s, sp<T>(L.k1)));
}

// EPL deflection, generic in the ray type. A ray inside rho < 1e-6 arcsec gets
// zero deflection (mask), computed without a branch so pairs stay in lockstep.
template <class T>
__device__ __forceinline__ void epl_fwd_T(const VecConst& V, const float* an, T x, T y, T& ax, T& ay) {
  const T dx = x - sp<T>(V.xc), dy = y - sp<T>(V.yc);
  // w = z - eps conj(z) = (dx - e1 dx - e2 dy, dy + e1 dy - e2 dx)
  const T wr = fmaT(sp<T>(-V.e1), dx, fmaT(sp<T>(-V.e2), dy, dx));
  const T wi = fmaT(sp<T>(V.e1), dy, fmaT(sp<T>(-V.e2), dx, dy));
  const T w2 = fmaT(wr, wr, wi * wi);
  const T keep = geT(w2, sp<T>(V.w2min));
  const T w2c = maxT(w2, sp<T>(V.w2min));   // > 0; where it clamps, keep = 0 zeroes the deflection
  const T S = keep * ex2T(fmaT(sp<T>(V.t), fmaT(sp<T>(-0.5f), lg2T(w2c), sp<T>(V.lc)), sp<T>(V.tlc_lo)));
  const T iw2 = rcpT(w2c);
  const T nwi = -wi;
  const T vr = fmaT(wr, wr, nwi * wi) * iw2;
  const T vi = sp<T>(2.f) * wr * wi * iw2;
  const T ur = fmaT(sp<T>(-V.e1), vr, sp<T>(-V.e2) * vi);
  const T ui = fmaT(sp<T>(V.e2), vr, sp<T>(-V.e1) * vi);
  const T nui = fmaT(sp<T>(-V.e2), vr, sp<T>(V.e1) * vi);   // -ui: packed FMAs take no negated operands
  // G = sum_{n<N} a_{n+1} u^n by Horner (g = a_n + u g), then F = 1 + u G
  T gr = sp<T>(0.f), gi = sp<T>(0.f);
#pragma unroll 2
  for (int n = V.nterms; n >= 1; --n) {
    const T ngr = fmaT(ur, gr, fmaT(nui, gi, sp<T>(an[n - 1])));
    gi = fmaT(ur, gi, ui * gr);
    gr = ngr;
  }
  const T hr = fmaT(ur, gr, fmaT(nui, gi, sp<T>(1.f)));
  const T hi = fmaT(ur, gi, ui * gr);
  ax = S * fmaT(wr, hr, nwi * hi);
  ay = S * fmaT(wr, hi, wi * hr);
}

template <class T>
__device__ __forceinline__ T ray_intensity_T(const VecConst& V, const float* an, T x, T y) {
  T ax, ay;
  epl_fwd_T(V, an, x, y, ax, ay);
  const T bx = x - ax - fmaT(sp<T>(V.g1), x, sp<T>(V.g2) * y);
  const T by = y - ay - fmaT(sp<T>(V.g2), x, sp<T>(-V.g1) * y);
  return sersic_fwd_T(V.light[1], bx, by) + sersic_fwd_T(V.light[0], x, y);
}

}  // namespace gl
