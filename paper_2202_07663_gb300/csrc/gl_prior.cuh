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


struct PriorTable {
  gl_prior_entry e[GL_NPARAM];
};

constexpr double kLnSqrt2Pi = 0.91893853320467274178;

// Bijector decided by the prior's support (Sec. 2.2): (0, inf) -> exp,
// (a, b) -> a + (b - a) sigmoid(z), R -> identity.
__device__ __forceinline__ void bij(const gl_prior_entry& e, double z, double& th, double& dth, double& lj,
                                    double& dlj) {
  if (e.kind == GL_PRIOR_LOGNORMAL) {
    th = exp(z);
    dth = th;
    lj = z;
    dlj = 1.0;
  } else if (e.kind == GL_PRIOR_TRUNCNORMAL || e.kind == GL_PRIOR_UNIFORM) {
    const double lo = e.kind == GL_PRIOR_UNIFORM ? e.a : e.c, hi = e.kind == GL_PRIOR_UNIFORM ? e.b : e.d;
    const double s = 1.0 / (1.0 + exp(-z));
    th = lo + (hi - lo) * s;
    dth = (hi - lo) * s * (1.0 - s);
    // log s + log(1 - s) = -softplus(-z) - softplus(z)
    const double sp_p = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
    const double sp_m = z > 0 ? log1p(exp(-z)) : -z + log1p(exp(z));
    lj = log(hi - lo) - sp_m - sp_p;
    dlj = 1.0 - 2.0 * s;
  } else {
    th = z;
    dth = 1.0;
    lj = 0.0;
    dlj = 0.0;
  }
}

__device__ __forceinline__ double inv_bij(const gl_prior_entry& e, double th) {
  if (e.kind == GL_PRIOR_LOGNORMAL) return log(th);
  if (e.kind == GL_PRIOR_TRUNCNORMAL || e.kind == GL_PRIOR_UNIFORM) {
    const double lo = e.kind == GL_PRIOR_UNIFORM ? e.a : e.c, hi = e.kind == GL_PRIOR_UNIFORM ? e.b : e.d;
    const double s = (th - lo) / (hi - lo);
    return log(s) - log1p(-s);
  }
  return th;
}

// log density of one prior marginal and its derivative (Eq. sim-dist).
__device__ __forceinline__ void logpdf(const gl_prior_entry& e, double x, double& lp, double& dlp) {
  switch (e.kind) {
    case GL_PRIOR_NORMAL: {
      const double r = (x - e.a) / e.b;
      lp = -0.5 * r * r - log(e.b) - kLnSqrt2Pi;
      dlp = -r / e.b;
      break;
    }
    case GL_PRIOR_LOGNORMAL: {
      const double r = (log(x) - log(e.a)) / e.b;
      lp = -0.5 * r * r - log(x) - log(e.b) - kLnSqrt2Pi;
      dlp = -r / (e.b * x) - 1.0 / x;
      break;
    }
    case GL_PRIOR_TRUNCNORMAL: {
      const double r = (x - e.a) / e.b;
      const double Z = 0.5 * (erf((e.d - e.a) / (e.b * 1.41421356237309504880)) -
                              erf((e.c - e.a) / (e.b * 1.41421356237309504880)));
      const bool in = x >= e.c && x <= e.d;
      lp = in ? -0.5 * r * r - log(e.b) - kLnSqrt2Pi - log(Z) : -INFINITY;
      dlp = -r / e.b;
      break;
    }
    default: {  // uniform
      const bool in = x >= e.a && x <= e.b;
      lp = in ? -log(e.b - e.a) : -INFINITY;
      dlp = 0.0;
    }
  }
}

// Copy and validate a caller's table of GL_NPARAM entries.
inline int load_table(const gl_prior_entry* prior, PriorTable& P) {
  if (!prior) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null prior");
  for (int j = 0; j < GL_NPARAM; ++j) {
    const gl_prior_entry& e = prior[j];
    const bool ok = (e.kind == GL_PRIOR_NORMAL && e.b > 0) || (e.kind == GL_PRIOR_LOGNORMAL && e.a > 0 && e.b > 0) ||
                    (e.kind == GL_PRIOR_TRUNCNORMAL && e.b > 0 && e.c < e.d) ||
                    (e.kind == GL_PRIOR_UNIFORM && e.a < e.b);
    if (!ok) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad prior entry");
    P.e[j] = e;
  }
  return GL_OK;
}

}  // namespace prior
}  // namespace gl
