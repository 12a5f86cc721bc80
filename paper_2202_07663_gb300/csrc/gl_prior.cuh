// gl_prior.cuh - the prior of the unconstrained parameters shared by MAP, HMC
// on the posterior and VI (arXiv:2202.07663, Sec. 2.2, Eq. sim-dist): the
// component-wise bijector chosen by each marginal's support, its inverse, and
// the log density of each marginal, FP64.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "../../include/gigalens.h"
#include "gl_internal.h"

namespace gl {
namespace prior {


// One marginal with the constants its functions need, computed once on the
// host (FP64 transcendentals are slow on GB300's narrow FP64 pipe):
// the support [lo, hi] and log(hi - lo) of the sigmoid bijector, 1/b, log a
// and the log normaliser (log b + log sqrt(2 pi), plus log of the truncated
// normal's mass in [c, d]; log(b - a) for the uniform).
struct PriorEntry {
  int kind;
  double a, b, c, d;
  double lo, hi, lwidth;
  double inv_b, log_a, lnorm;
};

struct PriorTable {
  PriorEntry e[GL_NPARAM];
};

constexpr double kLnSqrt2Pi = 0.91893853320467274178;

// Bijector decided by the prior's support (Sec. 2.2): (0, inf) -> exp,
// (a, b) -> a + (b - a) sigmoid(z), R -> identity. For the sigmoid, with
// e = exp(-|z|): s = 1/(1 + e) or e/(1 + e), and log s + log(1 - s) =
// -softplus(z) - softplus(-z) = -|z| - 2 log1p(e).
__device__ __forceinline__ void bij(const PriorEntry& e, double z, double& th, double& dth, double& lj,
                                    double& dlj) {
  if (e.kind == GL_PRIOR_LOGNORMAL) {
    th = exp(z);
    dth = th;
    lj = z;
    dlj = 1.0;
  } else if (e.kind == GL_PRIOR_TRUNCNORMAL || e.kind == GL_PRIOR_UNIFORM) {
    const double ez = exp(-fabs(z));
    const double s = z >= 0 ? 1.0 / (1.0 + ez) : ez / (1.0 + ez);
    th = e.lo + (e.hi - e.lo) * s;
    dth = (e.hi - e.lo) * s * (1.0 - s);
    lj = e.lwidth - fabs(z) - 2.0 * log1p(ez);
    dlj = 1.0 - 2.0 * s;
  } else {
    th = z;
    dth = 1.0;
    lj = 0.0;
    dlj = 0.0;
  }
}

__device__ __forceinline__ double inv_bij(const PriorEntry& e, double th) {
  if (e.kind == GL_PRIOR_LOGNORMAL) return log(th);
  if (e.kind == GL_PRIOR_TRUNCNORMAL || e.kind == GL_PRIOR_UNIFORM) {
    const double s = (th - e.lo) / (e.hi - e.lo);
    return log(s) - log1p(-s);
  }
  return th;
}

// log density of one prior marginal and its derivative (Eq. sim-dist).
__device__ __forceinline__ void logpdf(const PriorEntry& e, double x, double& lp, double& dlp) {
  switch (e.kind) {
    case GL_PRIOR_NORMAL: {
      const double r = (x - e.a) * e.inv_b;
      lp = -0.5 * r * r - e.lnorm;
      dlp = -r * e.inv_b;
      break;
    }
    case GL_PRIOR_LOGNORMAL: {
      const double lx = log(x);
      const double r = (lx - e.log_a) * e.inv_b;
      lp = -0.5 * r * r - lx - e.lnorm;
      dlp = -(r * e.inv_b + 1.0) / x;
      break;
    }
    case GL_PRIOR_TRUNCNORMAL: {
      const double r = (x - e.a) * e.inv_b;
      const bool in = x >= e.c && x <= e.d;
      lp = in ? -0.5 * r * r - e.lnorm : -INFINITY;
      dlp = -r * e.inv_b;
      break;
    }
    default: {  // uniform
      const bool in = x >= e.a && x <= e.b;
      lp = in ? -e.lnorm : -INFINITY;
      dlp = 0.0;
    }
  }
}

// Copy and validate a caller's table of GL_NPARAM entries and derive the
// per-marginal constants.
inline int load_table(const gl_prior_entry* prior, PriorTable& P) {
  if (!prior) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null prior");
  for (int j = 0; j < GL_NPARAM; ++j) {
    const gl_prior_entry& e = prior[j];
    const bool ok = (e.kind == GL_PRIOR_NORMAL && e.b > 0) || (e.kind == GL_PRIOR_LOGNORMAL && e.a > 0 && e.b > 0) ||
                    (e.kind == GL_PRIOR_TRUNCNORMAL && e.b > 0 && e.c < e.d) ||
                    (e.kind == GL_PRIOR_UNIFORM && e.a < e.b);
    if (!ok) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad prior entry");
    PriorEntry& q = P.e[j];
    q.kind = e.kind;
    q.a = e.a;
    q.b = e.b;
    q.c = e.c;
    q.d = e.d;
    q.lo = e.kind == GL_PRIOR_UNIFORM ? e.a : e.c;
    q.hi = e.kind == GL_PRIOR_UNIFORM ? e.b : e.d;
    q.lwidth = (e.kind == GL_PRIOR_UNIFORM || e.kind == GL_PRIOR_TRUNCNORMAL) ? std::log(q.hi - q.lo) : 0.0;
    q.inv_b = e.kind == GL_PRIOR_UNIFORM ? 0.0 : 1.0 / e.b;
    q.log_a = e.kind == GL_PRIOR_LOGNORMAL ? std::log(e.a) : 0.0;
    if (e.kind == GL_PRIOR_UNIFORM) {
      q.lnorm = std::log(e.b - e.a);
    } else {
      q.lnorm = std::log(e.b) + kLnSqrt2Pi;
      if (e.kind == GL_PRIOR_TRUNCNORMAL) {
        const double Z = 0.5 * (std::erf((e.d - e.a) / (e.b * 1.41421356237309504880)) -
                                std::erf((e.c - e.a) / (e.b * 1.41421356237309504880)));
        q.lnorm += std::log(Z);
      }
    }
  }
  return GL_OK;
}

}  // namespace prior
}  // namespace gl
