// FP64 CPU oracle for the GIGA-Lens forward model, log-likelihood and gradient
// (Gu, Huang et al., arXiv:2202.07663, Sec. 2.1 and 2.2).
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
// statement of what the GPU path computes. Only the tests, the smoke check and
// the CPU-baseline leg of the benchmark may load it. It shares no code, header,
// table or constant generator with the CUDA library and includes none of it.
//
// Every step follows the paper's own formulation, in the paper's order:
//   * ellipticity (e1, e2) -> (q, phi)                         Sec. 2.1.1, Eq. for (e1, e2)
//   * rotation into the profile frame                          Sec. 2.1.1, Eq. coord-trans
//   * EPL deflection by the Tessore & Metcalf (2015) series    Sec. 2.1.1 (EPL paragraph)
//   * external shear                                           Sec. 2.1.1, Eq. alpha_ext
//   * ray trace + surface-brightness conservation + lens light Sec. 2.1.1 (first paragraph)
//   * elliptical Sersic with b_n = 1.9992 n - 0.3271           Sec. 2.1.1, Eq. Sersic
//   * k x k supersampling, then averaging down                 Sec. 2.1.1 (last paragraph)
//   * times the pixel area: counts/s per pixel                 (reading below)
//   * PSF convolution                                          Sec. 2.1.1 (first paragraph)
//   * Gaussian log-likelihood with model-dependent variance    Sec. 2.1.2, Eq. model-def
//   * gradient of log L with respect to the 22 parameters      Sec. 2.2 (the paper uses AD;
//     here forward-mode dual numbers carried through the same code)
//
// Readings where the paper is silent (each also listed in the design notes):
//   * pixel centres are symmetric about (0, 0); x grows with the column index,
//     y with the row index; subpixel centres of the k-times finer grid likewise;
//   * the shear of Eq. alpha_ext acts about the image origin (0, 0);
//   * the lens-frame deflection is rotated back by the inverse of Eq. coord-trans;
//   * the convolution is a true convolution (kernel flipped), zero padded,
//     output the size of the input, odd K with centre (K-1)/2;
//   * phi = 0 when e1 = e2 = 0;
//   * inside the elliptical radius rho = sqrt(q x^2 + y^2/q) < 1e-6 arcsec the
//     EPL deflection is set to zero and the Sersic radius is floored at 1e-6;
//   * the series is summed until a term (value and every derivative) falls
//     below 1e-18 in magnitude; the summed function is O(1);
//   * the amplitudes I_l, I_s are surface brightness in counts/s/arcsec^2 and a
//     detector pixel records the flux falling on it, counts/s: the mean over
//     its k x k subpixels times the pixel area (pixel scale squared). The
//     paper's simulated sample (I_l ~ 300, I_s ~ 150, sigma_bkg = 0.2 counts/s,
//     HST-like, Sec. 3) and the posterior widths behind its Table 3 fit this
//     reading; sampling the brightness without the area would make those
//     images about 240 times brighter per pixel.
//
// Parameter order (Table 2): thetaE, gamma_epl, e_epl1, e_epl2, x_epl, y_epl,
// gamma_ext1, gamma_ext2, R_l, n_l, e_l1, e_l2, x_l, y_l, I_l,
// R_s, n_s, e_s1, e_s2, x_s, y_s, I_s.

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NPARAM = 22;
constexpr double RHO_MIN = 1e-6;       // arcsec
constexpr double SERIES_TOL = 1e-18;   // absolute, on value and derivatives
constexpr int SERIES_CAP = 100000;
constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Forward-mode dual numbers: value plus ND directional derivatives.
// ---------------------------------------------------------------------------
template <int ND>
struct Dual {
  double v;
  double d[ND];
  Dual() : v(0.0) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }  // NOLINT
};

template <int ND>
inline Dual<ND> chain(const Dual<ND>& x, double f, double dfdx) {
  Dual<ND> r;
  r.v = f;
  for (int i = 0; i < ND; ++i) r.d[i] = dfdx * x.d[i];
  return r;
}

template <int ND> inline Dual<ND> operator+(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v + b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int ND> inline Dual<ND> operator-(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v - b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int ND> inline Dual<ND> operator-(const Dual<ND>& a) {
  Dual<ND> r; r.v = -a.v; for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r;
}
template <int ND> inline Dual<ND> operator*(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v * b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int ND> inline Dual<ND> operator/(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v / b.v;
  const double inv = 1.0 / b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
template <int ND> inline Dual<ND> operator+(const Dual<ND>& a, double b) { Dual<ND> r = a; r.v += b; return r; }
template <int ND> inline Dual<ND> operator+(double a, const Dual<ND>& b) { return b + a; }
template <int ND> inline Dual<ND> operator-(const Dual<ND>& a, double b) { Dual<ND> r = a; r.v -= b; return r; }
template <int ND> inline Dual<ND> operator-(double a, const Dual<ND>& b) { return -(b - a); }
template <int ND> inline Dual<ND> operator*(const Dual<ND>& a, double b) {
  Dual<ND> r; r.v = a.v * b; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b; return r;
}
template <int ND> inline Dual<ND> operator*(double a, const Dual<ND>& b) { return b * a; }
template <int ND> inline Dual<ND> operator/(const Dual<ND>& a, double b) { return a * (1.0 / b); }
template <int ND> inline Dual<ND> operator/(double a, const Dual<ND>& b) { return Dual<ND>(a) / b; }
template <int ND> inline Dual<ND>& operator+=(Dual<ND>& a, const Dual<ND>& b) { a = a + b; return a; }

template <int ND> inline Dual<ND> sqrt(const Dual<ND>& x) { const double s = std::sqrt(x.v); return chain(x, s, 0.5 / s); }
template <int ND> inline Dual<ND> exp(const Dual<ND>& x) { const double e = std::exp(x.v); return chain(x, e, e); }
template <int ND> inline Dual<ND> log(const Dual<ND>& x) { return chain(x, std::log(x.v), 1.0 / x.v); }
template <int ND> inline Dual<ND> cos(const Dual<ND>& x) { return chain(x, std::cos(x.v), -std::sin(x.v)); }
template <int ND> inline Dual<ND> sin(const Dual<ND>& x) { return chain(x, std::sin(x.v), std::cos(x.v)); }
template <int ND> inline Dual<ND> pow(const Dual<ND>& x, const Dual<ND>& y) { return exp(y * log(x)); }
template <int ND> inline Dual<ND> atan2(const Dual<ND>& y, const Dual<ND>& x) {
  Dual<ND> r;
  r.v = std::atan2(y.v, x.v);
  const double den = x.v * x.v + y.v * y.v;
  for (int i = 0; i < ND; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / den;
  return r;
}

inline double val(double x) { return x; }
template <int ND> inline double val(const Dual<ND>& x) { return x.v; }
inline double mag(double x) { return std::fabs(x); }
template <int ND> inline double mag(const Dual<ND>& x) {
  double m = std::fabs(x.v);
  for (int i = 0; i < ND; ++i) m = std::fmax(m, std::fabs(x.d[i]));
  return m;
}
using std::atan2; using std::cos; using std::exp; using std::log; using std::pow; using std::sin; using std::sqrt;

template <class T> struct Cx { T re, im; };
template <class T> inline Cx<T> cmul(const Cx<T>& a, const Cx<T>& b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// ---------------------------------------------------------------------------
// Model pieces, generic in the scalar type (double or Dual<22>).
// ---------------------------------------------------------------------------

// Sec. 2.1.1: (e1, e2) = (1-q)/(1+q) (cos 2phi, sin 2phi), inverted.
template <class T>
void ellipticity_to_q_phi(const T& e1, const T& e2, T& q, T& phi) {
  if (val(e1) == 0.0 && val(e2) == 0.0) {  // phi undefined: take phi = 0, q = 1
    q = T(1.0);
    phi = T(0.0);
    return;
  }
  const T e = sqrt(e1 * e1 + e2 * e2);
  q = (1.0 - e) / (1.0 + e);
  phi = 0.5 * atan2(e2, e1);
}

// Sec. 2.1.1, Eq. coord-trans: image frame -> profile frame.
template <class T>
void to_profile_frame(const T& x, const T& y, const T& xc, const T& yc, const T& phi, T& xp, T& yp) {
  const T c = cos(phi), s = sin(phi);
  const T dx = x - xc, dy = y - yc;
  xp = c * dx + s * dy;
  yp = -s * dx + c * dy;
}

// Tessore & Metcalf (2015) angular function, as cited in Sec. 2.1.1:
//   Omega = sum_n Omega_n,  Omega_0 = e^{i phi_ell},
//   Omega_n = -f (2n - (2-t)) / (2n + (2-t)) e^{2 i phi_ell} Omega_{n-1},
// with f = (1-q)/(1+q). nterms < 0 sums to convergence; otherwise exactly
// terms n = 0..nterms-1 are summed.
template <class T>
Cx<T> epl_omega(const Cx<T>& eiphi, const T& f, const T& t, int nterms) {
  const Cx<T> e2iphi = cmul(eiphi, eiphi);
  Cx<T> term = eiphi;
  Cx<T> sum = eiphi;
  const int cap = nterms < 0 ? SERIES_CAP : nterms;
  for (int n = 1; n < cap; ++n) {
    const T cn = -f * (2.0 * n - (2.0 - t)) / (2.0 * n + (2.0 - t));
    term = cmul(Cx<T>{cn * e2iphi.re, cn * e2iphi.im}, term);
    sum.re += term.re;
    sum.im += term.im;
    if (nterms < 0 && mag(term.re) < SERIES_TOL && mag(term.im) < SERIES_TOL) break;
  }
  return sum;
}

// EPL deflection (Sec. 2.1.1): convergence
//   kappa = (3-gamma)/2 (thetaE / sqrt(q x_l^2 + y_l^2/q))^(gamma-1),
// i.e. Tessore & Metcalf's kappa = (2-t)/2 (b/R)^t with t = gamma-1,
// b = thetaE sqrt(q), R = sqrt(q^2 x_l^2 + y_l^2); deflection in the lens frame
//   alpha = 2b/(1+q) (b/R)^(t-1) Omega(phi_ell),  e^{i phi_ell} = (q x_l + i y_l)/R,
// rotated back to the image frame.
template <class T>
void epl_deflection(const T& x, const T& y, const T* m, T& ax, T& ay, int nterms = -1) {
  const T& thetaE = m[0];
  const T& gamma = m[1];
  T q, phi;
  ellipticity_to_q_phi(m[2], m[3], q, phi);
  T xl, yl;
  to_profile_frame(x, y, m[4], m[5], phi, xl, yl);
  const double rho_v = std::sqrt(val(q) * val(xl) * val(xl) + val(yl) * val(yl) / val(q));
  if (rho_v < RHO_MIN) {
    ax = T(0.0);
    ay = T(0.0);
    return;
  }
  const T t = gamma - 1.0;
  const T b = thetaE * sqrt(q);
  const T R = sqrt(q * q * xl * xl + yl * yl);
  const Cx<T> eiphi{q * xl / R, yl / R};
  const T f = (1.0 - q) / (1.0 + q);
  const Cx<T> om = epl_omega(eiphi, f, t, nterms);
  const T pref = 2.0 * b / (1.0 + q) * pow(b / R, t - 1.0);
  const T alx = pref * om.re, aly = pref * om.im;
  const T c = cos(phi), s = sin(phi);
  ax = c * alx - s * aly;
  ay = s * alx + c * aly;
}

// External shear (Sec. 2.1.1, Eq. alpha_ext), about the image origin.
template <class T>
void shear_deflection(const T& x, const T& y, const T& g1, const T& g2, T& ax, T& ay) {
  ax = g1 * x + g2 * y;
  ay = g2 * x - g1 * y;
}

// Elliptical Sersic (Sec. 2.1.1, Eq. Sersic) with b_n = 1.9992 n - 0.3271.
// l = (R_eff, n, e1, e2, xc, yc, I0).
template <class T>
T sersic(const T& x, const T& y, const T* l) {
  T q, phi;
  ellipticity_to_q_phi(l[2], l[3], q, phi);
  T xl, yl;
  to_profile_frame(x, y, l[4], l[5], phi, xl, yl);
  T rho = sqrt(q * xl * xl + yl * yl / q);
  if (val(rho) < RHO_MIN) rho = T(RHO_MIN);
  const T bn = 1.9992 * l[1] - 0.3271;
  return l[6] * exp(-bn * (pow(rho / l[0], 1.0 / l[1]) - 1.0));
}

// Ray trace to the source plane (lens equation): beta = theta - alpha_epl - alpha_ext.
template <class T>
void ray_trace(double x, double y, const T* p, T& bx, T& by) {
  T ax, ay, sx, sy;
  epl_deflection(T(x), T(y), p, ax, ay);
  shear_deflection(T(x), T(y), p[6], p[7], sx, sy);
  bx = x - ax - sx;
  by = y - ay - sy;
}

// Surface brightness at an image-plane point: lensed source (surface
// brightness conservation) plus lens light, Sec. 2.1.1.
template <class T>
T surface_brightness(double x, double y, const T* p) {
  T bx, by;
  ray_trace(x, y, p, bx, by);
  return sersic(bx, by, p + 15) + sersic(T(x), T(y), p + 8);
}

// Supersampled grid, averaged down by k (Sec. 2.1.1, last paragraph).
template <class T>
void binned_image(const T* p, int H, int W, int k, double dpix, T* out) {
  const double sub = dpix / k;
  const double cx = (k * W - 1) * 0.5, cy = (k * H - 1) * 0.5;
  for (int i = 0; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      T acc(0.0);
      for (int a = 0; a < k; ++a) {
        for (int b = 0; b < k; ++b) {
          const double x = (j * k + b - cx) * sub;
          const double y = (i * k + a - cy) * sub;
          acc += surface_brightness(x, y, p);
        }
      }
      out[i * W + j] = acc / double(k * k);
    }
  }
}

// True 2-D convolution, zero padding, output the size of the input.
template <class T>
void convolve(const T* img, int H, int W, const double* psf, int K, T* out) {
  const int c = (K - 1) / 2;
  for (int i = 0; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      T acc(0.0);
      for (int a = 0; a < K; ++a) {
        const int ii = i + c - a;
        if (ii < 0 || ii >= H) continue;
        for (int b = 0; b < K; ++b) {
          const int jj = j + c - b;
          if (jj < 0 || jj >= W) continue;
          acc += psf[a * K + b] * img[ii * W + jj];
        }
      }
      out[i * W + j] = acc;
    }
  }
}

struct System {
  const double* image;   // [H, W] observed, counts/s
  const double* sigma;   // [H, W] background noise std-dev
  int H, W;
  const double* psf;     // [K, K]
  int K;
  double dpix;           // arcsec per detector pixel
  int k;                 // supersampling factor
  double gain_exposure;  // G * t_exp; <= 0 drops the Poisson term
};

// Sec. 2.1.2, Eq. model-def.
template <class T>
void likelihood(const System& s, const T* model, T& ll, T& chi2) {
  ll = T(0.0);
  chi2 = T(0.0);
  for (int i = 0; i < s.H * s.W; ++i) {
    T var = T(s.sigma[i] * s.sigma[i]);
    if (s.gain_exposure > 0.0) var = var + model[i] / s.gain_exposure;
    const T r = s.image[i] - model[i];
    const T c2 = r * r / var;
    chi2 += c2;
    ll += -0.5 * (c2 + log(2.0 * PI * var));
  }
}

template <class T>
void model_image(const System& s, const T* p, std::vector<T>& pre, std::vector<T>& model) {
  pre.assign(size_t(s.H) * s.W, T(0.0));
  model.assign(size_t(s.H) * s.W, T(0.0));
  binned_image(p, s.H, s.W, s.k, s.dpix, pre.data());
  const double area = s.dpix * s.dpix;
  for (size_t i = 0; i < pre.size(); ++i) pre[i] = pre[i] * area;
  convolve(pre.data(), s.H, s.W, s.psf, s.K, model.data());
}

int set_threads(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

}  // namespace

extern "C" {

// Number of threads OpenMP would use for nthreads <= 0.
int orc_max_threads() { return set_threads(0); }

// EPL deflection at n points. m = (thetaE, gamma, e1, e2, xc, yc).
// nterms < 0: series to convergence; otherwise exactly nterms terms.
void orc_epl_deflection(const double* x, const double* y, long n, const double* m, int nterms,
                        double* ax, double* ay) {
  for (long i = 0; i < n; ++i) epl_deflection(x[i], y[i], m, ax[i], ay[i], nterms);
}

// Tessore & Metcalf angular function Omega at the elliptical angle phi_ell.
void orc_epl_omega(double phi_ell, double q, double t, int nterms, double* re, double* im) {
  const Cx<double> e{std::cos(phi_ell), std::sin(phi_ell)};
  const Cx<double> om = epl_omega(e, (1.0 - q) / (1.0 + q), t, nterms);
  *re = om.re;
  *im = om.im;
}

void orc_shear_deflection(const double* x, const double* y, long n, double g1, double g2,
                          double* ax, double* ay) {
  for (long i = 0; i < n; ++i) shear_deflection(x[i], y[i], g1, g2, ax[i], ay[i]);
}

// l = (R_eff, n, e1, e2, xc, yc, I0).
void orc_sersic(const double* x, const double* y, long n, const double* l, double* out) {
  for (long i = 0; i < n; ++i) out[i] = sersic(x[i], y[i], l);
}

void orc_ray_trace(const double* x, const double* y, long n, const double* p, double* bx, double* by) {
  for (long i = 0; i < n; ++i) ray_trace(x[i], y[i], p, bx[i], by[i]);
}

void orc_surface_brightness(const double* x, const double* y, long n, const double* p, double* out) {
  for (long i = 0; i < n; ++i) out[i] = surface_brightness(x[i], y[i], p);
}

// Binned (pre-PSF) image of one parameter vector.
void orc_binned_image(const double* p, int H, int W, int k, double dpix, double* out) {
  binned_image(p, H, W, k, dpix, out);
}

void orc_convolve(const double* img, int H, int W, const double* psf, int K, double* out) {
  convolve(img, H, W, psf, K, out);
}

// log L and chi^2 (Sec. 2.1.2, Eq. model-def) of a given model image.
void orc_likelihood_image(const double* model, const double* image, const double* sigma, int H, int W,
                          double gain_exposure, double* loglik, double* chi2) {
  const System s{image, sigma, H, W, nullptr, 0, 0.0, 1, gain_exposure};
  likelihood(s, model, *loglik, *chi2);
}

// Model image M [H, W] and its Jacobian J [H, W, 22] = dM / d params of one
// vector (forward-mode duals through binning and convolution).
void orc_model_jacobian(const double* params, int H, int W, const double* psf, int K, double dpix, int k,
                        double* model_out, double* jac_out) {
  const System s{nullptr, nullptr, H, W, psf, K, dpix, k, 0.0};
  using D = Dual<NPARAM>;
  D p[NPARAM];
  for (int i = 0; i < NPARAM; ++i) {
    p[i] = D(params[i]);
    p[i].d[i] = 1.0;
  }
  std::vector<D> pre, model;
  model_image(s, p, pre, model);
  for (int i = 0; i < H * W; ++i) {
    model_out[i] = model[i].v;
    for (int j = 0; j < NPARAM; ++j) jac_out[size_t(i) * NPARAM + j] = model[i].d[j];
  }
}

// Noiseless model images (PSF-convolved) for B parameter vectors: out [B, H, W].
void orc_simulate(const double* params, int B, int H, int W, const double* psf, int K,
                  double dpix, int k, double* out, int nthreads) {
  const System s{nullptr, nullptr, H, W, psf, K, dpix, k, 0.0};
  const int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic) num_threads(nt)
  for (int b = 0; b < B; ++b) {
    std::vector<double> pre, model;
    model_image(s, params + size_t(b) * NPARAM, pre, model);
    std::memcpy(out + size_t(b) * H * W, model.data(), sizeof(double) * H * W);
  }
}

// log L and chi^2 for B vectors; grad [B, 22] (d log L / d params) when non-null.
void orc_loglik(const double* params, int B, const double* image, const double* sigma, int H, int W,
                const double* psf, int K, double dpix, int k, double gain_exposure,
                double* loglik, double* chi2, double* grad, int nthreads) {
  const System s{image, sigma, H, W, psf, K, dpix, k, gain_exposure};
  const int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic) num_threads(nt)
  for (int b = 0; b < B; ++b) {
    const double* pb = params + size_t(b) * NPARAM;
    if (grad == nullptr) {
      std::vector<double> pre, model;
      model_image(s, pb, pre, model);
      double ll, c2;
      likelihood(s, model.data(), ll, c2);
      if (loglik) loglik[b] = ll;
      if (chi2) chi2[b] = c2;
    } else {
      using D = Dual<NPARAM>;
      D p[NPARAM];
      for (int i = 0; i < NPARAM; ++i) {
        p[i] = D(pb[i]);
        p[i].d[i] = 1.0;
      }
      std::vector<D> pre, model;
      model_image(s, p, pre, model);
      D ll, c2;
      likelihood(s, model.data(), ll, c2);
      if (loglik) loglik[b] = ll.v;
      if (chi2) chi2[b] = c2.v;
      for (int i = 0; i < NPARAM; ++i) grad[size_t(b) * NPARAM + i] = ll.d[i];
    }
  }
}

}  // extern "C"
