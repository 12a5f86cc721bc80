"""FP64 oracle of the variant likelihood (arXiv:2202.07663, Sec. 2.1.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). The paper mentions an
alternative variance map built from the observed image,
sigma_tot^2 = sigma_bkg^2 + I_obs / (G t_exp), independent of the parameters,
with negative observed pixels set to zero (its footnote on lenstronomy). The
model is then linear in the two light amplitudes, M = I_l A_l + I_s A_s with
A_l, A_s the model images at unit amplitude, so for the other parameters the
amplitudes that maximise log L solve the 2x2 weighted least-squares system

  [<A_l, A_l>  <A_l, A_s>] [I_l]   [<A_l, D>]
  [<A_s, A_l>  <A_s, A_s>] [I_s] = [<A_s, D>],   <a, b> = sum a b / sigma_tot^2,

and log L profiled over them is a function of the other 20 parameters.
Where the system is singular (an amplitude whose image is zero on the
detector, to 1e-12 of the other's weighted self-product, or two images
proportional to 1e-12 of det), the amplitude with the smaller self-product is
0 and the other is solved alone.
The gradient of the profiled log L in the remaining parameters is the
gradient of log L at the solved amplitudes (they are a stationary point).
Everything else comes from the model oracle.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _model

I_L, I_S = 14, 21
SINGULAR = 1e-12   # relative size below which a self-product or determinant counts as zero


def observed_variance(image, sigma_bkg, gain_exposure: float):
    """sigma_bkg^2 + max(I_obs, 0) / (G t_exp), per pixel."""
    image = np.asarray(image, np.float64)
    s2 = np.broadcast_to(np.asarray(sigma_bkg, np.float64) ** 2, image.shape)
    if gain_exposure > 0:
        return s2 + np.maximum(image, 0.0) / gain_exposure
    return np.array(s2)


def basis_images(params, H, W, psf, pixel_scale, k):
    """Model images at (I_l, I_s) = (1, 0) and (0, 1): [B, 2, H, W]."""
    p = np.atleast_2d(np.asarray(params, np.float64))
    pl, ps = p.copy(), p.copy()
    pl[:, I_L], pl[:, I_S] = 1.0, 0.0
    ps[:, I_L], ps[:, I_S] = 0.0, 1.0
    Al = _model.simulate(pl, H, W, psf, pixel_scale, k)
    As = _model.simulate(ps, H, W, psf, pixel_scale, k)
    return np.stack([Al, As], axis=1)


def solve_amplitudes(A, image, var):
    """(I_l, I_s) per vector from basis images A [B, 2, H, W]."""
    D = np.asarray(image, np.float64)
    w = 1.0 / np.asarray(var, np.float64)
    out = np.zeros((A.shape[0], 2))
    for b in range(A.shape[0]):
        G = np.array([[np.sum(w * A[b, i] * A[b, j]) for j in range(2)] for i in range(2)])
        r = np.array([np.sum(w * A[b, i] * D) for i in range(2)])
        gmax = max(G[0, 0], G[1, 1])
        live = [i for i in range(2) if G[i, i] > SINGULAR * gmax]
        if len(live) == 2 and np.linalg.det(G) > SINGULAR * G[0, 0] * G[1, 1]:
            out[b] = np.linalg.solve(G, r)
        elif live:
            # singular: keep the amplitude with the larger self-product, zero the other
            i = max(live, key=lambda j: G[j, j])
            out[b, i] = r[i] / G[i, i]
    return out


def profiled_loglik(params, image, sigma_bkg, psf, pixel_scale, k, gain_exposure, grad=True):
    """(log L, chi^2, grad [B, 22], amplitudes [B, 2]) of the variant likelihood
    profiled over (I_l, I_s); the gradient's amplitude entries are set to 0."""
    p = np.atleast_2d(np.asarray(params, np.float64)).copy()
    H, W = np.asarray(image).shape
    var = observed_variance(image, sigma_bkg, gain_exposure)
    A = basis_images(p, H, W, psf, pixel_scale, k)
    amps = solve_amplitudes(A, image, var)
    p[:, I_L], p[:, I_S] = amps[:, 0], amps[:, 1]
    ll, c2, g = _model.loglik(p, image, np.sqrt(var), psf, pixel_scale, k, 0.0, grad=True)
    if grad:
        g = g.copy()
        g[:, I_L] = 0.0
        g[:, I_S] = 0.0
    return ll, c2, (g if grad else None), amps
