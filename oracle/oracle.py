"""ctypes wrapper around the FP64 CPU oracle (``gl_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the oracle is the plain statement of what the GPU
path computes (arXiv:2202.07663, Sec. 2.1-2.2). Only ``tests/``, the smoke
check and the CPU-baseline leg of ``bench.py`` may import it. The product
package never imports this module, and this module imports nothing from the
product package.

Every array crossing this boundary is float64, C-contiguous. Parameter vectors
are rows of 22 values in the order of Table 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gl_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
# A test may point the loader at a deliberately broken build of the oracle
# (mutation testing of the pins); nothing else sets this.
_LIB_OVERRIDE = os.environ.get("GL_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

NPARAM = 22

_d = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP); returns the library path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        i, l = ctypes.c_int, ctypes.c_long
        dbl = ctypes.c_double
        sig = {
            "orc_max_threads": ([], i),
            "orc_epl_deflection": ([_d, _d, l, _d, i, _d, _d], None),
            "orc_epl_omega": ([dbl, dbl, dbl, i, _d, _d], None),
            "orc_shear_deflection": ([_d, _d, l, dbl, dbl, _d, _d], None),
            "orc_sersic": ([_d, _d, l, _d, _d], None),
            "orc_ray_trace": ([_d, _d, l, _d, _d, _d], None),
            "orc_surface_brightness": ([_d, _d, l, _d, _d], None),
            "orc_binned_image": ([_d, i, i, i, dbl, _d], None),
            "orc_convolve": ([_d, i, i, _d, i, _d], None),
            "orc_simulate": ([_d, i, i, i, _d, i, dbl, i, _d, i], None),
            "orc_model_jacobian": ([_d, i, i, _d, i, dbl, i, _d, _d], None),
            "orc_likelihood_image": ([_d, _d, _d, i, i, dbl, _d, _d], None),
            "orc_loglik": ([_d, i, _d, _d, i, i, _d, i, dbl, i, dbl, _d, _d, _d, i], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_d)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def epl_deflection(x, y, mass, nterms: int = -1):
    """EPL deflection (alpha_x, alpha_y) at points; mass = (thetaE, gamma, e1, e2, xc, yc)."""
    x, y = np.broadcast_arrays(_f64(x), _f64(y))
    x, y = _f64(x), _f64(y)
    m = _f64(mass)
    ax, ay = np.empty_like(x), np.empty_like(x)
    _load().orc_epl_deflection(_p(x), _p(y), x.size, _p(m), int(nterms), _p(ax), _p(ay))
    return ax, ay


def epl_omega(phi_ell: float, q: float, t: float, nterms: int = -1) -> complex:
    """Tessore & Metcalf angular series Omega(phi_ell) for axis ratio q and t = gamma - 1."""
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_epl_omega(float(phi_ell), float(q), float(t), int(nterms), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def shear_deflection(x, y, g1: float, g2: float):
    x, y = np.broadcast_arrays(_f64(x), _f64(y))
    x, y = _f64(x), _f64(y)
    ax, ay = np.empty_like(x), np.empty_like(x)
    _load().orc_shear_deflection(_p(x), _p(y), x.size, float(g1), float(g2), _p(ax), _p(ay))
    return ax, ay


def sersic(x, y, light):
    """Elliptical Sersic at points; light = (R_eff, n, e1, e2, xc, yc, I0)."""
    x, y = np.broadcast_arrays(_f64(x), _f64(y))
    x, y = _f64(x), _f64(y)
    l = _f64(light)
    out = np.empty_like(x)
    _load().orc_sersic(_p(x), _p(y), x.size, _p(l), _p(out))
    return out


def ray_trace(x, y, params):
    x, y = np.broadcast_arrays(_f64(x), _f64(y))
    x, y = _f64(x), _f64(y)
    p = _f64(params)
    bx, by = np.empty_like(x), np.empty_like(x)
    _load().orc_ray_trace(_p(x), _p(y), x.size, _p(p), _p(bx), _p(by))
    return bx, by


def surface_brightness(x, y, params):
    x, y = np.broadcast_arrays(_f64(x), _f64(y))
    x, y = _f64(x), _f64(y)
    p = _f64(params)
    out = np.empty_like(x)
    _load().orc_surface_brightness(_p(x), _p(y), x.size, _p(p), _p(out))
    return out


def binned_image(params, H: int, W: int, k: int, pixel_scale: float) -> np.ndarray:
    p = _f64(params)
    out = np.empty((H, W), dtype=np.float64)
    _load().orc_binned_image(_p(p), H, W, k, float(pixel_scale), _p(out))
    return out


def convolve(img, psf) -> np.ndarray:
    img, psf = _f64(img), _f64(psf)
    H, W = img.shape
    K = psf.shape[0]
    out = np.empty_like(img)
    _load().orc_convolve(_p(img), H, W, _p(psf), K, _p(out))
    return out


def simulate(params, H: int, W: int, psf, pixel_scale: float, k: int, nthreads: int = 0) -> np.ndarray:
    """Noiseless PSF-convolved model images, [B, H, W]."""
    p = _f64(params).reshape(-1, NPARAM)
    psf = _f64(psf)
    B = p.shape[0]
    out = np.empty((B, H, W), dtype=np.float64)
    _load().orc_simulate(_p(p), B, H, W, _p(psf), psf.shape[0], float(pixel_scale), int(k), _p(out), int(nthreads))
    return out


def loglik(params, image, sigma, psf, pixel_scale: float, k: int, gain_exposure: float,
           grad: bool = False, nthreads: int = 0):
    """(loglik[B], chi2[B], grad[B,22] or None) per Sec. 2.1.2 Eq. model-def."""
    p = _f64(params).reshape(-1, NPARAM)
    image, sigma, psf = _f64(image), _f64(sigma), _f64(psf)
    if sigma.shape != image.shape:
        sigma = _f64(np.broadcast_to(sigma, image.shape))
    H, W = image.shape
    B = p.shape[0]
    ll = np.empty(B)
    c2 = np.empty(B)
    g = np.empty((B, NPARAM)) if grad else None
    _load().orc_loglik(_p(p), B, _p(image), _p(sigma), H, W, _p(psf), psf.shape[0], float(pixel_scale),
                       int(k), float(gain_exposure), _p(ll), _p(c2), _p(g) if grad else None, int(nthreads))
    return ll, c2, g


def likelihood_image(model, image, sigma, gain_exposure: float):
    """(log L, chi^2) of a given model image, Sec. 2.1.2 Eq. model-def."""
    model, image = _f64(model), _f64(image)
    sigma = _f64(np.broadcast_to(_f64(sigma), image.shape))
    H, W = image.shape
    ll, c2 = ctypes.c_double(), ctypes.c_double()
    _load().orc_likelihood_image(_p(model), _p(image), _p(sigma), H, W, float(gain_exposure),
                                 ctypes.byref(ll), ctypes.byref(c2))
    return ll.value, c2.value


def model_jacobian(params, H: int, W: int, psf, pixel_scale: float, k: int):
    """(M [H, W], J [H, W, 22]): model image of one vector and dM/dparams."""
    p = _f64(params).reshape(NPARAM)
    psf = _f64(psf)
    M = np.empty((H, W))
    J = np.empty((H, W, NPARAM))
    _load().orc_model_jacobian(_p(p), H, W, _p(psf), psf.shape[0], float(pixel_scale), int(k), _p(M), _p(J))
    return M, J
