"""Seeded synthetic inputs for the lens-likelihood hot path.

This module holds input generation only: parameter draws, PSF images, noise
realisations and the serving request stream. It contains none of the lens
model's arithmetic (no deflection, no light profile, no convolution, no
likelihood), so both the CUDA path and the FP64 oracle may use it.

Parameter vectors have 22 entries in the order of Table 2 of arXiv:2202.07663:
  0 thetaE   1 gamma_epl  2 e_epl1  3 e_epl2  4 x_epl  5 y_epl
  6 gamma_ext1  7 gamma_ext2
  8 R_l  9 n_l  10 e_l1  11 e_l2  12 x_l  13 y_l  14 I_l
  15 R_s  16 n_s  17 e_s1  18 e_s2  19 x_s  20 y_s  21 I_s
Units: arcsec for positions and radii, counts/s for amplitudes.

The paper's 100 lenstronomy systems and its TinyTim PSF are not available;
these synthetic systems stand in for them with the paper's pixel scale
(0.065 arcsec, Sec. 3) and the distributions below.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

NPARAM = 22
PARAM_NAMES = (
    "theta_E", "gamma_epl", "e_epl1", "e_epl2", "x_epl", "y_epl",
    "gamma_ext1", "gamma_ext2",
    "R_l", "n_l", "e_l1", "e_l2", "x_l", "y_l", "I_l",
    "R_s", "n_s", "e_s1", "e_s2", "x_s", "y_s", "I_s",
)

PIXEL_SCALE = 0.065  # arcsec per detector pixel (Sec. 3)

# Box used for multi-start draws and for clipping perturbed vectors: the truth
# ranges of the uniform parameters and +-2 sigma of the normal ones.
PRIOR_BOX = np.array([
    [1.0, 2.0],      # theta_E
    [1.8, 2.2],      # gamma_epl
    [-0.2, 0.2],     # e_epl1
    [-0.2, 0.2],     # e_epl2
    [-0.1, 0.1],     # x_epl
    [-0.1, 0.1],     # y_epl
    [-0.1, 0.1],     # gamma_ext1
    [-0.1, 0.1],     # gamma_ext2
    [0.5, 1.5],      # R_l
    [2.0, 5.0],      # n_l
    [-0.2, 0.2],     # e_l1
    [-0.2, 0.2],     # e_l2
    [-0.1, 0.1],     # x_l
    [-0.1, 0.1],     # y_l
    [100.0, 1000.0],  # I_l
    [0.05, 0.3],     # R_s
    [0.5, 4.0],      # n_s
    [-0.3, 0.3],     # e_s1
    [-0.3, 0.3],     # e_s2
    [-0.6, 0.6],     # x_s
    [-0.6, 0.6],     # y_s
    [50.0, 500.0],   # I_s
], dtype=np.float64)


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    """Shape and noise model of one synthetic lens system."""
    H: int
    W: int
    k: int                      # supersampling factor
    K: int                      # PSF side (odd)
    psf: str = "gaussian"       # "gaussian" (FWHM 0.1") or "moffat" (beta 3, FWHM 0.12")
    pixel_scale: float = PIXEL_SCALE
    sigma_bkg: float = 0.01
    gain_exposure: float = 1000.0   # G * t_exp, seconds (G = 1)


# The fixed-shape workloads: shapes, PSFs, batch sizes and the base of their
# seeds (system s of a workload draws from PCG64 seeded with seed + s).
PLAIN = "plain-60x60-k2-psf11-B64"
MULTISTART = "multistart-60x60-k2-psf11-B4096"
HMC = "hmc-100x100-k4-moffat21-B512"
STRESS = "stress-200x200-k4-psf21-B16384"
WORKLOADS = {
    PLAIN: dict(spec=SystemSpec(60, 60, 2, 11, "gaussian"), B=64, draw="perturbed", seed=1000),
    MULTISTART: dict(spec=SystemSpec(60, 60, 2, 11, "gaussian"), B=4096, draw="box", seed=2000),
    HMC: dict(spec=SystemSpec(100, 100, 4, 21, "moffat"), B=512, draw="perturbed", seed=3000),
    STRESS: dict(spec=SystemSpec(200, 200, 4, 21, "gaussian"), B=16384, draw="box", seed=5000),
}


def rng_for(workload: str, system: int = 0) -> np.random.Generator:
    """PCG64 stream of system ``system`` of a workload: seed = its base + system."""
    return np.random.default_rng(WORKLOADS[workload]["seed"] + system)


def draw_truth(rng: np.random.Generator) -> np.ndarray:
    """One truth vector from the synthetic simulation distribution."""
    p = np.empty(NPARAM)
    p[0] = rng.uniform(1.0, 2.0)
    p[1] = rng.uniform(1.8, 2.2)
    p[2:4] = rng.normal(0.0, 0.1, 2)
    p[4:6] = rng.normal(0.0, 0.05, 2)
    p[6:8] = rng.normal(0.0, 0.05, 2)
    p[8] = rng.uniform(0.5, 1.5)
    p[9] = rng.uniform(2.0, 5.0)
    p[10:12] = rng.normal(0.0, 0.1, 2)
    p[12:14] = rng.normal(0.0, 0.05, 2)
    p[14] = math.exp(rng.uniform(math.log(100.0), math.log(1000.0)))
    p[15] = rng.uniform(0.05, 0.3)
    p[16] = rng.uniform(0.5, 4.0)
    p[17:19] = rng.normal(0.0, 0.15, 2)
    p[19:21] = p[4:6] + rng.normal(0.0, 0.3, 2)
    p[21] = math.exp(rng.uniform(math.log(50.0), math.log(500.0)))
    return p


def draw_perturbed(rng: np.random.Generator, truth: np.ndarray, B: int, frac: float = 0.02) -> np.ndarray:
    """B vectors: truth + N(0, frac * box width), clipped to the box."""
    width = PRIOR_BOX[:, 1] - PRIOR_BOX[:, 0]
    out = truth[None, :] + rng.normal(0.0, 1.0, (B, NPARAM)) * (frac * width)[None, :]
    lo = np.minimum(PRIOR_BOX[:, 0], truth)
    hi = np.maximum(PRIOR_BOX[:, 1], truth)
    return np.clip(out, lo, hi)


def draw_box(rng: np.random.Generator, B: int) -> np.ndarray:
    """B multi-start vectors, uniform over the box (amplitudes log-uniform)."""
    u = rng.uniform(0.0, 1.0, (B, NPARAM))
    out = PRIOR_BOX[:, 0] + u * (PRIOR_BOX[:, 1] - PRIOR_BOX[:, 0])
    for j in (14, 21):
        lo, hi = np.log(PRIOR_BOX[j])
        out[:, j] = np.exp(lo + u[:, j] * (hi - lo))
    return out


def gaussian_psf(K: int, fwhm: float = 0.1, pixel_scale: float = PIXEL_SCALE) -> np.ndarray:
    """Gaussian PSF sampled at pixel centres, normalised to unit sum."""
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0))) / pixel_scale
    c = (K - 1) / 2.0
    r = np.arange(K) - c
    g = np.exp(-0.5 * (r[:, None] ** 2 + r[None, :] ** 2) / sig ** 2)
    return g / g.sum()


def moffat_psf(K: int, beta: float = 3.0, fwhm: float = 0.12, pixel_scale: float = PIXEL_SCALE) -> np.ndarray:
    """Moffat PSF sampled at pixel centres, normalised to unit sum."""
    alpha = fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0)) / pixel_scale
    c = (K - 1) / 2.0
    r = np.arange(K) - c
    m = (1.0 + (r[:, None] ** 2 + r[None, :] ** 2) / alpha ** 2) ** (-beta)
    return m / m.sum()


def make_psf(spec: SystemSpec) -> np.ndarray:
    if spec.psf == "gaussian":
        return gaussian_psf(spec.K, pixel_scale=spec.pixel_scale)
    if spec.psf == "moffat":
        return moffat_psf(spec.K, pixel_scale=spec.pixel_scale)
    raise ValueError("unknown psf kind %r" % spec.psf)


def add_noise(rng: np.random.Generator, model: np.ndarray, sigma_bkg: float, gain_exposure: float) -> np.ndarray:
    """Observed image from a noiseless model image (counts/s):
    Poisson(G t_exp M) / (G t_exp) + N(0, sigma_bkg^2)."""
    model = np.asarray(model, dtype=np.float64)
    out = model.copy()
    if gain_exposure > 0:
        out = rng.poisson(np.clip(model, 0.0, None) * gain_exposure) / gain_exposure
    return out + rng.normal(0.0, sigma_bkg, model.shape)


# The paper's simulation distribution and (broader) prior, Eq. sim-dist
# (Sec. 2.1.2), as samplers: ("n", mu, sd), ("ln", median, sd of log),
# ("tn", mu, sd, lo, hi), ("u", lo, hi). Used to draw synthetic systems and
# multi-start initial points; the methods evaluate their own densities.
PAPER_SIM = [
    ("ln", 1.25, 0.25), ("tn", 2.0, 0.25, 1.0, 3.0), ("n", 0.0, 0.1), ("n", 0.0, 0.1), ("n", 0.0, 0.03),
    ("n", 0.0, 0.03), ("n", 0.0, 0.05), ("n", 0.0, 0.05),
    ("ln", 1.6, 0.15), ("u", 2.0, 6.0), ("tn", 0.0, 0.05, -0.15, 0.15), ("tn", 0.0, 0.05, -0.15, 0.15),
    ("n", 0.0, 0.01), ("n", 0.0, 0.01), ("ln", 300.0, 0.3),
    ("ln", 0.25, 0.15), ("u", 0.5, 4.0), ("tn", 0.0, 0.15, -0.5, 0.5), ("tn", 0.0, 0.15, -0.5, 0.5),
    ("n", 0.0, 0.25), ("n", 0.0, 0.25), ("ln", 150.0, 0.5),
]
PAPER_PRIOR_DRAW = [
    ("ln", 1.25, 0.4), ("tn", 2.0, 0.5, 1.0, 3.0), ("n", 0.0, 0.2), ("n", 0.0, 0.2), ("n", 0.0, 0.06),
    ("n", 0.0, 0.06), ("n", 0.0, 0.1), ("n", 0.0, 0.1),
    ("ln", 1.6, 0.25), ("u", 0.5, 8.0), ("tn", 0.0, 0.1, -0.15, 0.15), ("tn", 0.0, 0.1, -0.15, 0.15),
    ("n", 0.0, 0.02), ("n", 0.0, 0.02), ("ln", 300.0, 0.5),
    ("ln", 0.25, 0.25), ("u", 0.5, 8.0), ("tn", 0.0, 0.3, -0.5, 0.5), ("tn", 0.0, 0.3, -0.5, 0.5),
    ("n", 0.0, 0.5), ("n", 0.0, 0.5), ("ln", 150.0, 0.9),
]

# Sec. 3 simulated sample: 80x80 pixels at 0.065", sigma_bkg 0.2, t_exp 100 s, G = 1, k = 2
PAPER_SAMPLE_SPEC = SystemSpec(80, 80, 2, 11, "gaussian", PIXEL_SCALE, 0.2, 100.0)


def draw_table(rng: np.random.Generator, table, n: int) -> np.ndarray:
    """n independent draws from a per-parameter distribution table."""
    out = np.empty((n, len(table)))
    for j, d in enumerate(table):
        kind = d[0]
        if kind == "n":
            out[:, j] = rng.normal(d[1], d[2], n)
        elif kind == "ln":
            out[:, j] = np.exp(rng.normal(math.log(d[1]), d[2], n))
        elif kind == "u":
            out[:, j] = rng.uniform(d[1], d[2], n)
        elif kind == "tn":
            col = np.empty(0)
            while col.size < n:   # rejection from the normal
                x = rng.normal(d[1], d[2], 4 * n)
                col = np.concatenate([col, x[(x >= d[3]) & (x <= d[4])]])
            out[:, j] = col[:n]
        else:
            raise ValueError(kind)
    return out


@dataclasses.dataclass
class LensRequest:
    """One request of the serving stream."""
    index: int
    arrival_s: float
    spec: SystemSpec
    B: int
    seed: int


def serving_stream(n: int = 1000, rate_hz: float = 20.0, seed: int = 4000,
                   sizes: Tuple[int, ...] = (40, 60, 80, 120), ks: Tuple[int, ...] = (2, 4),
                   Ks: Tuple[int, ...] = (11, 21), bmin: int = 256, bmax: int = 2048) -> List[LensRequest]:
    """Seeded Poisson arrivals of heterogeneous lens systems."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    out = []
    for i in range(n):
        s = int(rng.choice(sizes))
        spec = SystemSpec(s, s, int(rng.choice(ks)), int(rng.choice(Ks)), "gaussian")
        out.append(LensRequest(i, float(t[i]), spec, int(rng.integers(bmin, bmax + 1)), seed * 1000 + i))
    return out
