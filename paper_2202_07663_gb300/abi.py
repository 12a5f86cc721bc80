"""ctypes binding of the C ABI in ``include/gigalens.h`` (same function names).

Argument marshalling only: every step of the likelihood runs in the CUDA
library ``csrc/libgigalens.so``. If the library is missing or cannot be
loaded, every call raises: there is no CPU fallback.

Torch tensors are passed by device pointer together with the current CUDA
stream of their device.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Sequence

import numpy as np

NPARAM = 22
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "libgigalens.so")

GL_OK = 0
GL_ERR_INVALID_ARG, GL_ERR_OOM, GL_ERR_CUDA, GL_ERR_TIMEOUT, GL_ERR_BUDGET, GL_ERR_UNSUPPORTED = range(-1, -7, -1)
GL_K_SETUP, GL_K_RAY_FWD, GL_K_CONV, GL_K_RAY_ADJ, GL_K_FINAL, GL_K_OTHER, GL_K_ORDER = range(7)
GL_KERNEL_KINDS = 7
GL_MAX_SEGMENTS = 256

_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_f = ctypes.c_float

# name -> (argtypes, restype), mirroring include/gigalens.h
SIGNATURES = {
    "gl_system_create": ([ctypes.POINTER(_vp), _vp, _vp, _f, _i, _i, _vp, _i, _d, _i, _d, _vp], _i),
    "gl_system_create_obsvar": ([ctypes.POINTER(_vp), _vp, _vp, _f, _i, _i, _vp, _i, _d, _i, _d, _vp], _i),
    "gl_system_destroy": ([_vp], _i),
    "gl_system_reserve": ([_vp, _i], _i),
    "gl_system_scratch_bytes": ([_vp, _i], ctypes.c_size_t),
    "gl_system_resident_bytes": ([_vp], ctypes.c_size_t),
    "gl_system_scratch_held": ([_vp], ctypes.c_size_t),
    "gl_loglik": ([_vp, _vp, _i, _vp, _vp, _vp], _i),
    "gl_loglik_grad": ([_vp, _vp, _i, _vp, _vp, _vp, _vp], _i),
    "gl_loglik_grad_host": ([_vp, _vp, _i, _vp, _vp, _vp, _vp], _i),
    "gl_simulate": ([_vp, _vp, _i, _vp, _vp], _i),
    "gl_loglik_grad_grouped": ([_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp], _i),
    "gl_loglik_grad_noalloc": ([_vp, _vp, _i, _vp, _vp, _vp, _vp], _i),
    "gl_batcher_create": ([ctypes.POINTER(_vp), _i, ctypes.c_size_t, _i, _i, _i], _i),
    "gl_batcher_destroy": ([_vp], _i),
    "gl_batcher_segment_bytes": ([_vp, _i], ctypes.c_size_t),
    "gl_batcher_run": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp], _i),
    "gl_map_inverse": ([_i, _vp, _vp, _vp, _vp], _i),
    "gl_map_transform": ([_i, _vp, _vp, _vp, _vp], _i),
    "gl_map_adam_step": ([_i, _vp, _vp, _vp, _i, _d, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_loglik_grad_profiled": ([_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_hmc_leapfrog": ([_i, _i, _vp, _vp, _vp, _vp, _d, _d, _vp, _vp], _i),
    "gl_hmc_leapfrog_dev": ([_i, _i, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp], _i),
    "gl_hmc_finish": ([_i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_hmc_chees": ([_i, _i, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp], _i),
    "gl_hmc_affine": ([_i, _i, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_hmc_affine_pullback": ([_i, _i, _vp, _vp, _vp, _vp], _i),
    "gl_vi_param_count": ([_i], ctypes.c_size_t),
    "gl_vi_workspace_bytes": ([_i, _i], ctypes.c_size_t),
    "gl_vi_sample": ([_i, _i, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_vi_step": ([_i, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _i, _d, _d, _d, _d, _vp, _vp, _vp, _vp], _i),
    "gl_vi_moments": ([_i, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp], _i),
    "gl_vi_apply": ([_i, _i, _i, _vp, _i, _vp, _vp, _vp, _i, _d, _d, _d, _d, _vp, _vp, _vp], _i),
    "gl_posterior_grad": ([_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_posterior_whitened_transform": ([_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_posterior_whitened_grad": ([_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_hmc_leapfrog_whitened": ([_i, _vp, _vp, _vp, _vp, _d, _vp, _d, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_hmc_leapfrog_whitened_chain": ([_i, _vp, _vp, _vp, _vp, _vp, _d, _vp, _d, _vp, _vp, _vp, _vp, _vp], _i),
    "gl_error_string": ([_i], ctypes.c_char_p),
    "gl_last_error_message": ([], ctypes.c_char_p),
    "gl_profile_enable": ([_i], _i),
    "gl_profile_reset": ([], _i),
    "gl_profile_read": ([_vp, _vp], _i),
    "gl_kernel_name": ([_i], ctypes.c_char_p),
    "gl_launch_count": ([], ctypes.c_longlong),
    "gl_profile_peak": ([_i, _vp], _i),
    "gl_psf_factor": ([_vp, _i, _vp, _i, _vp], _i),
    "gl_profile_select": ([ctypes.c_uint], _i),
    "gl_system_psf_rank": ([_vp], _i),
}


class PriorEntry(ctypes.Structure):
    """gl_prior_entry of include/gigalens.h."""
    _fields_ = [("kind", ctypes.c_int), ("reserved", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("c", ctypes.c_double), ("d", ctypes.c_double)]


GL_PRIOR_NORMAL, GL_PRIOR_LOGNORMAL, GL_PRIOR_TRUNCNORMAL, GL_PRIOR_UNIFORM = range(4)


class GLError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = lib_handle()
        msg = "%s: %s (%s)" % (where, lib.gl_error_string(code).decode(), lib.gl_last_error_message().decode())
        super().__init__(msg)
        self.code = code


def lib_handle():
    """Load the CUDA library (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("CUDA library %s is not built; run paper_2202_07663_gb300.build.build()" % LIB_PATH)
            lib = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(code: int, where: str) -> None:
    if code != GL_OK:
        raise GLError(code, where)


def _stream_ptr(device=None) -> int:
    import torch
    return torch.cuda.current_stream(device).cuda_stream


def _dptr(t, dtype, shape=None, name="tensor") -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be on a CUDA device" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return t.data_ptr()


# ------------------------------------------------------------- raw calls ----

def gl_system_create(image, noise_map, sigma_bkg, psf, pixel_scale, supersample, gain_exposure, stream=0,
                     observed_variance: bool = False):
    lib = lib_handle()
    create = lib.gl_system_create_obsvar if observed_variance else lib.gl_system_create
    image = np.ascontiguousarray(image, dtype=np.float32)
    psf = np.ascontiguousarray(psf, dtype=np.float32)
    H, W = image.shape
    K = psf.shape[0]
    if psf.shape != (K, K):
        raise ValueError("psf must be square")
    nm = None
    if noise_map is not None:
        nm = np.ascontiguousarray(np.broadcast_to(np.asarray(noise_map, dtype=np.float32), image.shape))
    h = _vp()
    code = create(ctypes.byref(h), image.ctypes.data, nm.ctypes.data if nm is not None else None,
                  float(sigma_bkg), H, W, psf.ctypes.data, K, float(pixel_scale), int(supersample),
                  float(gain_exposure), stream)
    _check(code, "gl_system_create_obsvar" if observed_variance else "gl_system_create")
    return h.value


def gl_system_destroy(handle) -> None:
    _check(lib_handle().gl_system_destroy(handle), "gl_system_destroy")


def gl_loglik(handle, params_ptr, B, loglik_ptr, chi2_ptr, stream):
    _check(lib_handle().gl_loglik(handle, params_ptr, B, loglik_ptr, chi2_ptr, stream), "gl_loglik")


def gl_loglik_grad(handle, params_ptr, B, loglik_ptr, chi2_ptr, grad_ptr, stream):
    _check(lib_handle().gl_loglik_grad(handle, params_ptr, B, loglik_ptr, chi2_ptr, grad_ptr, stream),
           "gl_loglik_grad")


def gl_loglik_grad_host(handle, params_ptr, B, loglik_ptr, chi2_ptr, grad_ptr, stream):
    _check(lib_handle().gl_loglik_grad_host(handle, params_ptr, B, loglik_ptr, chi2_ptr, grad_ptr, stream),
           "gl_loglik_grad_host")


def gl_simulate(handle, params_ptr, B, images_ptr, stream):
    _check(lib_handle().gl_simulate(handle, params_ptr, B, images_ptr, stream), "gl_simulate")


def gl_hmc_leapfrog(B, d, q, p, grad, inv_mass, eps, kick, q32, stream):
    _check(lib_handle().gl_hmc_leapfrog(B, d, q, p, grad, inv_mass, float(eps), float(kick), q32, stream),
           "gl_hmc_leapfrog")


def gl_hmc_leapfrog_dev(B, d, q, p, grad, inv_mass, eps_dev, kick, q32, stream):
    _check(lib_handle().gl_hmc_leapfrog_dev(B, d, q, p, grad, inv_mass, eps_dev, float(kick), q32, stream),
           "gl_hmc_leapfrog_dev")


def gl_hmc_finish(B, d, p0, logp0, p, grad_new, logp_new, q_new, inv_mass, log_u, eps, q, logp, grad, accepted,
                  stream, accept_prob=None):
    _check(lib_handle().gl_hmc_finish(B, d, p0, logp0, p, grad_new, logp_new, q_new, inv_mass, log_u, float(eps), q,
                                      logp, grad, accepted, accept_prob, stream), "gl_hmc_finish")


def gl_hmc_chees(B, d, q_prev, q_prop, p_prop, inv_mass, accept_prob, t, out, stream):
    _check(lib_handle().gl_hmc_chees(B, d, q_prev, q_prop, p_prop, inv_mass, accept_prob, float(t), out, stream),
           "gl_hmc_chees")


def gl_hmc_affine(B, d, x, mu, L, z, z32, stream):
    _check(lib_handle().gl_hmc_affine(B, d, x, mu, L, z, z32, stream), "gl_hmc_affine")


def gl_hmc_affine_pullback(B, d, grad_z, L, grad_x, stream):
    _check(lib_handle().gl_hmc_affine_pullback(B, d, grad_z, L, grad_x, stream), "gl_hmc_affine_pullback")


def gl_profile_enable(on: bool) -> None:
    lib_handle().gl_profile_enable(1 if on else 0)


def gl_profile_select(kinds) -> None:
    """Bracket only the given kernel kinds (an iterable of GL_K_* values)
    while profiling is on."""
    mask = 0
    for k in kinds:
        mask |= 1 << int(k)
    lib_handle().gl_profile_select(mask)


def gl_profile_reset() -> None:
    lib_handle().gl_profile_reset()


def gl_profile_read():
    """{kernel name: (launches, total ms)} since the last reset."""
    lib = lib_handle()
    n = (ctypes.c_longlong * GL_KERNEL_KINDS)()
    t = (ctypes.c_double * GL_KERNEL_KINDS)()
    lib.gl_profile_read(ctypes.addressof(n), ctypes.addressof(t))
    return {lib.gl_kernel_name(i).decode(): (int(n[i]), float(t[i])) for i in range(GL_KERNEL_KINDS)}


def gl_launch_count() -> int:
    return int(lib_handle().gl_launch_count())


GL_PEAK_FP32_FMA, GL_PEAK_MUFU_EX2 = 0, 1


def psf_factor(psf):
    """The PSF's separable terms as gl_system_create uses them: (R, fac) with
    fac [R, 2, K] (row factor sigma_r u_r, column factor v_r); R = 0 when
    the 2-D convolution is kept."""
    p = np.ascontiguousarray(psf, dtype=np.float32)
    K = p.shape[0]
    if p.shape != (K, K):
        raise ValueError("psf must be square")
    fac = np.zeros(2 * K * K, np.float32)
    r = ctypes.c_int()
    _check(lib_handle().gl_psf_factor(p.ctypes.data, K, fac.ctypes.data, fac.size, ctypes.addressof(r)),
           "gl_psf_factor")
    R = int(r.value)
    return R, fac[:2 * R * K].reshape(R, 2, K).copy()


def gl_profile_peak(kind: int) -> float:
    """Measured rate of a pipe of the current device: FP32 flop/s
    (GL_PEAK_FP32_FMA) or ex2 results/s (GL_PEAK_MUFU_EX2)."""
    r = ctypes.c_double()
    _check(lib_handle().gl_profile_peak(kind, ctypes.addressof(r)), "gl_profile_peak")
    return float(r.value)


# ------------------------------------------------------------ objects -------

class GLSystem:
    """A lens system resident on the current CUDA device.

    image, noise map and PSF are copied to the device once; the methods take
    and return torch CUDA tensors and run on the current stream.
    """

    def __init__(self, image, psf, pixel_scale: float, supersample: int, gain_exposure: float,
                 noise_map=None, sigma_bkg: float = 0.0, observed_variance: bool = False):
        import torch
        self.H, self.W = np.asarray(image).shape
        self.K = np.asarray(psf).shape[0]
        self.k = int(supersample)
        self.pixel_scale = float(pixel_scale)
        self.gain_exposure = float(gain_exposure)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.observed_variance = bool(observed_variance)
        self._h = gl_system_create(image, noise_map, sigma_bkg, psf, pixel_scale, supersample, gain_exposure,
                                   _stream_ptr(), observed_variance=observed_variance)

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            gl_system_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, B: int) -> None:
        _check(lib_handle().gl_system_reserve(self._h, int(B)), "gl_system_reserve")

    def scratch_bytes(self, B: int) -> int:
        return int(lib_handle().gl_system_scratch_bytes(self._h, int(B)))

    def resident_bytes(self) -> int:
        return int(lib_handle().gl_system_resident_bytes(self._h))

    def psf_rank(self) -> int:
        """Separable PSF terms the convolution uses (0: the 2-D stencil)."""
        r = int(lib_handle().gl_system_psf_rank(self._h))
        if r < 0:
            _check(r, "gl_system_psf_rank")
        return r

    def scratch_held(self) -> int:
        """Device bytes of scratch the system holds now (0 until a call needs some)."""
        return int(lib_handle().gl_system_scratch_held(self._h))

    def _params(self, params):
        import torch
        if params.dim() != 2 or params.shape[1] != NPARAM:
            raise ValueError("params must be [B, 22]")
        return _dptr(params, torch.float32, name="params"), params.shape[0]

    def loglik(self, params, chi2: bool = False, out=None):
        import torch
        p, B = self._params(params)
        if out is None:
            ll = torch.empty(B, dtype=torch.float64, device=params.device)
        else:
            ll = out
        c2 = torch.empty(B, dtype=torch.float64, device=params.device) if chi2 else None
        gl_loglik(self._h, p, B, _dptr(ll, torch.float64, (B,), "loglik"), c2.data_ptr() if chi2 else None,
                  _stream_ptr(params.device))
        return (ll, c2) if chi2 else ll

    def loglik_grad(self, params, chi2: bool = False, out=None):
        import torch
        p, B = self._params(params)
        if out is None:
            ll = torch.empty(B, dtype=torch.float64, device=params.device)
            g = torch.empty(B, NPARAM, dtype=torch.float64, device=params.device)
            c2 = torch.empty(B, dtype=torch.float64, device=params.device) if chi2 else None
        else:
            ll, g, c2 = out
        gl_loglik_grad(self._h, p, B, _dptr(ll, torch.float64, (B,), "loglik"),
                       _dptr(c2, torch.float64, (B,), "chi2") if c2 is not None else None,
                       _dptr(g, torch.float64, (B, NPARAM), "grad"), _stream_ptr(params.device))
        return (ll, g, c2) if chi2 else (ll, g)

    def loglik_grad_profiled(self, params, grad: bool = True, chi2: bool = False):
        """log L profiled over (I_l, I_s): (loglik [B], grad [B, 22] or None,
        amplitudes [B, 2][, chi2 [B]]); grad entries 14 and 21 are 0."""
        import torch
        p, B = self._params(params)
        dev = params.device
        ll = torch.empty(B, dtype=torch.float64, device=dev)
        g = torch.empty(B, NPARAM, dtype=torch.float64, device=dev) if grad else None
        amps = torch.empty(B, 2, dtype=torch.float64, device=dev)
        c2 = torch.empty(B, dtype=torch.float64, device=dev) if chi2 else None
        _check(lib_handle().gl_loglik_grad_profiled(self._h, p, B, ll.data_ptr(),
                                                    c2.data_ptr() if chi2 else None,
                                                    g.data_ptr() if grad else None, amps.data_ptr(),
                                                    _stream_ptr(dev)), "gl_loglik_grad_profiled")
        return (ll, g, amps, c2) if chi2 else (ll, g, amps)

    def loglik_grad_host(self, params: np.ndarray, loglik: np.ndarray, grad: np.ndarray, chi2=None) -> None:
        """Host-buffer path: params float32 [B,22] and outputs float64 host arrays
        (pinned memory is fastest). Synchronous."""
        B = params.shape[0]
        for a, dt, shp in ((params, np.float32, (B, NPARAM)), (loglik, np.float64, (B,)),
                           (grad, np.float64, (B, NPARAM))):
            if a.dtype != dt or a.shape != shp or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host buffer must be %s %s contiguous" % (dt, shp))
        gl_loglik_grad_host(self._h, params.ctypes.data, B, loglik.ctypes.data,
                            chi2.ctypes.data if chi2 is not None else None, grad.ctypes.data, _stream_ptr())

    def simulate(self, params):
        import torch
        p, B = self._params(params)
        out = torch.empty(B, self.H, self.W, dtype=torch.float32, device=params.device)
        gl_simulate(self._h, p, B, out.data_ptr(), _stream_ptr(params.device))
        return out


def loglik_grad_grouped(systems: Sequence[GLSystem], params: Sequence, grad: bool = True, chi2: bool = False):
    """One grouped launch over several systems; returns lists (loglik, grad, chi2)."""
    import torch
    n = len(systems)
    if n < 1 or n > GL_MAX_SEGMENTS:
        raise ValueError("1..%d segments" % GL_MAX_SEGMENTS)
    lls, grads, c2s = [], [], []
    hs = (_vp * n)(*[s.handle for s in systems])
    pp = (_vp * n)()
    bb = (_i * n)()
    lp = (_vp * n)()
    gp = (_vp * n)()
    cp = (_vp * n)()
    dev = params[0].device
    for i, (s, p) in enumerate(zip(systems, params)):
        ptr, B = s._params(p)
        ll = torch.empty(B, dtype=torch.float64, device=dev)
        g = torch.empty(B, NPARAM, dtype=torch.float64, device=dev) if grad else None
        c2 = torch.empty(B, dtype=torch.float64, device=dev) if chi2 else None
        lls.append(ll)
        grads.append(g)
        c2s.append(c2)
        pp[i], bb[i], lp[i] = ptr, B, ll.data_ptr()
        gp[i] = g.data_ptr() if grad else None
        cp[i] = c2.data_ptr() if chi2 else None
    code = lib_handle().gl_loglik_grad_grouped(ctypes.addressof(hs), ctypes.addressof(pp), ctypes.addressof(bb),
                                               ctypes.addressof(lp), ctypes.addressof(cp) if chi2 else None,
                                               ctypes.addressof(gp) if grad else None, n, _stream_ptr(dev))
    _check(code, "gl_loglik_grad_grouped")
    return lls, grads, c2s


class Batcher:
    """Graph-replayed grouped launches over (system, vector range) segments."""

    def __init__(self, max_segments: int, arena_bytes: int, max_H: int, max_W: int, max_K: int):
        h = _vp()
        _check(lib_handle().gl_batcher_create(ctypes.byref(h), int(max_segments), int(arena_bytes), int(max_H),
                                              int(max_W), int(max_K)), "gl_batcher_create")
        self._h = h.value
        self.max_segments = int(max_segments)
        self.arena_bytes = int(arena_bytes)

    @staticmethod
    def segment_bytes(system: GLSystem, B: int) -> int:
        return int(lib_handle().gl_batcher_segment_bytes(system.handle, int(B)))

    def run(self, systems, params_ptrs, Bs, loglik_ptrs, grad_ptrs, stream=None) -> None:
        """One batch. params/loglik/grad are device pointers (ints) per segment."""
        import torch
        n = len(systems)
        hs = (_vp * n)(*[s.handle for s in systems])
        pp = (_vp * n)(*params_ptrs)
        bb = (_i * n)(*Bs)
        lp = (_vp * n)(*loglik_ptrs)
        gp = (_vp * n)(*grad_ptrs)
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib_handle().gl_batcher_run(self._h, ctypes.addressof(hs), ctypes.addressof(pp), ctypes.addressof(bb),
                                           ctypes.addressof(lp), None, ctypes.addressof(gp), n, st),
               "gl_batcher_run")

    def close(self) -> None:
        if getattr(self, "_h", None):
            _check(lib_handle().gl_batcher_destroy(self._h), "gl_batcher_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
