"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks one piece of the oracle against something other than the
oracle itself: closed forms, limits, invariants, library routines, statements
printed in arXiv:2202.07663 and brute-force relations. Together they are
chosen so that a dropped term, a wrong sign or index, or a transposed operand
anywhere in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, signal, special, stats

import oracle
from paper_2202_07663_gb300 import inputs

RNG = np.random.default_rng(12345)


def _e_from_q(q, phi=0.0):
    f = (1.0 - q) / (1.0 + q)
    return f * math.cos(2 * phi), f * math.sin(2 * phi)


# ---------------------------------------------------------------- EPL -------

@pytest.mark.parametrize("q", [0.3, 0.5, 0.7, 0.95])
def test_epl_matches_closed_form_sie_at_gamma_2(q):
    """gamma = 2 is the singular isothermal ellipsoid; its deflection for
    kappa = thetaE / (2 sqrt(q x^2 + y^2/q)) has the closed form (Kormann et
    al. 1994; Keeton 2001) alpha_x = thetaE sqrt(q)/s atan(s x/psi),
    alpha_y = thetaE sqrt(q)/s atanh(s y/psi), s = sqrt(1-q^2), psi = sqrt(q^2 x^2 + y^2)."""
    thetaE, xc, yc = 1.37, 0.04, -0.03
    e1, e2 = _e_from_q(q)
    x = RNG.uniform(-3, 3, 200)
    y = RNG.uniform(-3, 3, 200)
    ax, ay = oracle.epl_deflection(x, y, [thetaE, 2.0, e1, e2, xc, yc])
    dx, dy = x - xc, y - yc
    s = math.sqrt(1 - q * q)
    psi = np.sqrt(q * q * dx * dx + dy * dy)
    ex = thetaE * math.sqrt(q) / s * np.arctan(s * dx / psi)
    ey = thetaE * math.sqrt(q) / s * np.arctanh(s * dy / psi)
    np.testing.assert_allclose(ax, ex, rtol=0, atol=1e-13)
    np.testing.assert_allclose(ay, ey, rtol=0, atol=1e-13)


@pytest.mark.parametrize("gamma", [1.3, 1.7, 2.0, 2.4, 2.8])
def test_epl_circular_power_law(gamma):
    """q = 1: Gauss's law gives |alpha| = M(<r)/(pi r) = thetaE^(gamma-1) r^(2-gamma), radial."""
    thetaE = 1.2
    x = RNG.uniform(-3, 3, 100)
    y = RNG.uniform(-3, 3, 100)
    ax, ay = oracle.epl_deflection(x, y, [thetaE, gamma, 0.0, 0.0, 0.0, 0.0])
    r = np.hypot(x, y)
    mag = thetaE ** (gamma - 1) * r ** (2 - gamma)
    np.testing.assert_allclose(ax, mag * x / r, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ay, mag * y / r, rtol=1e-13, atol=1e-15)


def test_epl_sis_has_constant_deflection():
    """gamma = 2, q = 1 (singular isothermal sphere): |alpha| = thetaE everywhere."""
    x = RNG.uniform(-3, 3, 100)
    y = RNG.uniform(-3, 3, 100)
    ax, ay = oracle.epl_deflection(x, y, [1.61, 2.0, 0.0, 0.0, 0.0, 0.0])
    np.testing.assert_allclose(np.hypot(ax, ay), 1.61, rtol=1e-14)


@pytest.mark.parametrize("q", [1.0, 0.6])
def test_epl_point_mass_limit(q):
    """gamma -> 3: the mass within any ellipse tends to pi thetaE^2 concentrated at
    the centre, so alpha -> thetaE^2 (x, y)/r^2 for every axis ratio."""
    thetaE = 1.1
    e1, e2 = _e_from_q(q, 0.3)
    x = RNG.uniform(0.5, 3, 50) * RNG.choice([-1, 1], 50)
    y = RNG.uniform(0.5, 3, 50) * RNG.choice([-1, 1], 50)
    ax, ay = oracle.epl_deflection(x, y, [thetaE, 3.0 - 1e-9, e1, e2, 0.0, 0.0])
    r2 = x * x + y * y
    np.testing.assert_allclose(ax, thetaE ** 2 * x / r2, rtol=1e-7)
    np.testing.assert_allclose(ay, thetaE ** 2 * y / r2, rtol=1e-7)


def _kappa(x, y, thetaE, gamma, e1, e2, xc, yc):
    """Convergence as printed in Sec. 2.1.1 (Eq. kappa with Eq. coord-trans)."""
    e = math.hypot(e1, e2)
    q = (1 - e) / (1 + e)
    phi = 0.5 * math.atan2(e2, e1)
    xl = math.cos(phi) * (x - xc) + math.sin(phi) * (y - yc)
    yl = -math.sin(phi) * (x - xc) + math.cos(phi) * (y - yc)
    return (3 - gamma) / 2 * (thetaE / np.sqrt(q * xl * xl + yl * yl / q)) ** (gamma - 1)


@pytest.mark.parametrize("seed", range(6))
def test_epl_divergence_is_twice_kappa_and_curl_free(seed):
    """Poisson equation: div alpha = 2 kappa; alpha is a gradient: curl alpha = 0."""
    rng = np.random.default_rng(seed)
    m = [rng.uniform(0.8, 2.0), rng.uniform(1.5, 2.6), rng.normal(0, 0.15), rng.normal(0, 0.15),
         rng.normal(0, 0.05), rng.normal(0, 0.05)]
    x = rng.uniform(-2.5, 2.5, 40)
    y = rng.uniform(-2.5, 2.5, 40)
    h = 1e-5
    axp, _ = oracle.epl_deflection(x + h, y, m)
    axm, _ = oracle.epl_deflection(x - h, y, m)
    _, ayp = oracle.epl_deflection(x, y + h, m)
    _, aym = oracle.epl_deflection(x, y - h, m)
    div = (axp - axm) / (2 * h) + (ayp - aym) / (2 * h)
    np.testing.assert_allclose(div, 2 * _kappa(x, y, *m), rtol=2e-7)
    _, ayxp = oracle.epl_deflection(x + h, y, m)
    _, ayxm = oracle.epl_deflection(x - h, y, m)
    axyp, _ = oracle.epl_deflection(x, y + h, m)
    axym, _ = oracle.epl_deflection(x, y - h, m)
    curl = (ayxp - ayxm) / (2 * h) - (axyp - axym) / (2 * h)
    assert np.max(np.abs(curl)) < 1e-6 * np.max(np.abs(div))


@pytest.mark.parametrize("gamma,q", [(1.6, 0.55), (2.0, 0.8), (2.3, 0.45), (1.9, 0.9)])
def test_epl_matches_homoeoid_quadrature(gamma, q):
    """Independent route to alpha for a homoeoidal kappa(xi), xi^2 = x^2 + y^2/q^2
    (Schramm 1990; Keeton 2001): alpha_x = q x J_0, alpha_y = q y J_1 with
    J_n = int_0^1 kappa(xi(u)) / (1 - (1-q^2) u)^(n+1/2) du,
    xi(u)^2 = u (x^2 + y^2 / (1 - (1-q^2) u)). Here kappa(xi) is the paper's
    kappa with q x^2 + y^2/q = q xi^2."""
    thetaE = 1.3
    e1, _ = _e_from_q(q)
    a = (gamma - 1) / 2

    def khat_reg(u, x, y):  # kappa(xi(u)) * u^a  (the u^-a singularity is the quad weight)
        d = 1 - (1 - q * q) * u
        xi2_over_u = x * x + y * y / d
        return (3 - gamma) / 2 * (thetaE / math.sqrt(q * xi2_over_u)) ** (gamma - 1)

    for x, y in [(0.7, 0.4), (-1.3, 0.9), (0.2, -1.8), (2.1, 1.1)]:
        J = []
        for n in (0, 1):
            f = lambda u: khat_reg(u, x, y) / (1 - (1 - q * q) * u) ** (n + 0.5)  # noqa: E731
            val, _ = integrate.quad(f, 0.0, 1.0, weight="alg", wvar=(-a, 0.0), epsabs=1e-14, epsrel=1e-13)
            J.append(val)
        ax, ay = oracle.epl_deflection(np.array([x]), np.array([y]), [thetaE, gamma, e1, 0.0, 0.0, 0.0])
        assert ax[0] == pytest.approx(q * x * J[0], rel=1e-10)
        assert ay[0] == pytest.approx(q * y * J[1], rel=1e-10)


@pytest.mark.parametrize("t,q", [(0.6, 0.5), (1.0, 0.7), (1.3, 0.4), (0.9, 0.95)])
def test_epl_series_is_gauss_hypergeometric(t, q):
    """Tessore & Metcalf: Omega(phi) = e^{i phi} 2F1(1, t/2; 2 - t/2; -f e^{2 i phi})."""
    mpmath = pytest.importorskip("mpmath")
    f = (1 - q) / (1 + q)
    for phi in np.linspace(-3.0, 3.0, 9):
        z = -f * complex(math.cos(2 * phi), math.sin(2 * phi))
        ref = complex(math.cos(phi), math.sin(phi)) * complex(mpmath.hyp2f1(1, t / 2, 2 - t / 2, z))
        got = oracle.epl_omega(phi, q, t)
        assert abs(got - ref) < 1e-14
        ref2 = complex(math.cos(phi), math.sin(phi)) * special.hyp2f1(1, t / 2, 2 - t / 2, z)
        assert abs(got - ref2) < 1e-12


def test_epl_series_truncation_statement(golden_constants):
    """Sec. 2.1.1: truncation error <~ 1e-16 within 35 iterations for q >~ 0.5."""
    q = golden_constants["epl_series_q"]
    n = int(golden_constants["epl_series_iterations"])
    tol = golden_constants["epl_series_error"]
    for t in (0.4, 0.8, 1.0, 1.2, 1.6):
        for phi in np.linspace(-1.5, 1.5, 7):
            full = oracle.epl_omega(phi, q, t)
            part = oracle.epl_omega(phi, q, t, nterms=n)
            assert abs(full - part) <= tol
            # and the series has not converged after far fewer terms
            assert abs(full - oracle.epl_omega(phi, q, t, nterms=3)) > 1e-6


def _rot(x, y, psi):
    c, s = math.cos(psi), math.sin(psi)
    return c * x - s * y, s * x + c * y


@pytest.mark.parametrize("psi", [0.4, -1.1, 2.5])
def test_epl_rotation_covariance(psi):
    """Rotating the lens (centre and position angle) rotates the deflection field:
    alpha'(R z) = R alpha(z) when (e1 + i e2) -> (e1 + i e2) e^{2 i psi}."""
    m = [1.3, 2.15, 0.12, -0.07, 0.05, -0.02]
    x = RNG.uniform(-2, 2, 30)
    y = RNG.uniform(-2, 2, 30)
    ax, ay = oracle.epl_deflection(x, y, m)
    e = complex(m[2], m[3]) * complex(math.cos(2 * psi), math.sin(2 * psi))
    xc, yc = _rot(m[4], m[5], psi)
    xr, yr = _rot(x, y, psi)
    bx, by = oracle.epl_deflection(xr, yr, [m[0], m[1], e.real, e.imag, xc, yc])
    ex, ey = _rot(ax, ay, psi)
    np.testing.assert_allclose(bx, ex, atol=1e-13)
    np.testing.assert_allclose(by, ey, atol=1e-13)


def test_epl_position_angle_sense():
    """e2 > 0 puts the major axis at +45 degrees: the convergence (div alpha / 2)
    at equal distance is larger along the major axis (x = y) than across it."""
    m = [1.2, 2.0, 0.0, 0.25, 0.0, 0.0]
    h, d = 1e-5, 1.0 / math.sqrt(2)

    def div(x, y):
        axp, _ = oracle.epl_deflection([x + h], [y], m)
        axm, _ = oracle.epl_deflection([x - h], [y], m)
        _, ayp = oracle.epl_deflection([x], [y + h], m)
        _, aym = oracle.epl_deflection([x], [y - h], m)
        return float((axp - axm + ayp - aym)[0] / (2 * h))

    assert div(d, d) > 1.3 * div(-d, d)


# -------------------------------------------------------------- shear -------

def test_shear_is_traceless_symmetric_with_printed_components():
    """External shear: the Jacobian of alpha_ext is [[g1, g2], [g2, -g1]]
    (convergence-free, curl-free, shear components g1 = (psi_xx - psi_yy)/2,
    g2 = psi_xy), checked by finite differences."""
    g1, g2 = 0.031, -0.047
    x = RNG.uniform(-3, 3, 20)
    y = RNG.uniform(-3, 3, 20)
    h = 1e-4
    axp, ayp = oracle.shear_deflection(x + h, y, g1, g2)
    axm, aym = oracle.shear_deflection(x - h, y, g1, g2)
    bxp, byp = oracle.shear_deflection(x, y + h, g1, g2)
    bxm, bym = oracle.shear_deflection(x, y - h, g1, g2)
    np.testing.assert_allclose((axp - axm) / (2 * h), g1, atol=1e-12)
    np.testing.assert_allclose((ayp - aym) / (2 * h), g2, atol=1e-12)
    np.testing.assert_allclose((bxp - bxm) / (2 * h), g2, atol=1e-12)
    np.testing.assert_allclose((byp - bym) / (2 * h), -g1, atol=1e-12)
    ax, ay = oracle.shear_deflection(np.zeros(1), np.zeros(1), g1, g2)
    assert ax[0] == 0 and ay[0] == 0  # acts about the image origin


# ------------------------------------------------------------- Sersic -------

def test_sersic_amplitude_and_bn_constants(golden_constants):
    """I(rho = R_eff) = I0 by construction; at rho -> 0, I -> I0 exp(b_n) with the
    paper's b_n = 1.9992 n - 0.3271 (Sec. 2.1.1)."""
    a = golden_constants["sersic_bn_slope"]
    c = golden_constants["sersic_bn_offset"]
    for n in (0.5, 1.0, 2.5, 4.0):
        R, I0 = 0.7, 123.0
        # along the major axis (phi = 0): rho = sqrt(q) x  =>  x = R / sqrt(q)
        e1 = 0.2
        q = (1 - e1) / (1 + e1)
        val = oracle.sersic([R / math.sqrt(q)], [0.0], [R, n, e1, 0.0, 0.0, 0.0, I0])[0]
        assert val == pytest.approx(I0, rel=1e-13)
        centre = oracle.sersic([0.0], [0.0], [R, n, 0.0, 0.0, 0.0, 0.0, I0])[0]
        bn = a * n - c
        assert math.log(centre / I0) == pytest.approx(bn * (1 - (1e-6 / R) ** (1 / n)), rel=1e-12)


@pytest.mark.parametrize("n,q", [(1.0, 1.0), (1.5, 0.6), (0.8, 0.8)])
def test_sersic_total_flux(n, q):
    """Total flux of the elliptical Sersic: 2 pi n R^2 I0 e^{b_n} Gamma(2n) / b_n^{2n},
    independent of q (the ellipse q x^2 + y^2/q = rho^2 has area pi rho^2)."""
    R, I0 = 0.25, 1.0
    e1, e2 = _e_from_q(q, 0.4)
    bn = 1.9992 * n - 0.3271
    expect = 2 * math.pi * n * R * R * I0 * math.exp(bn) * math.gamma(2 * n) / bn ** (2 * n)
    L, N = 12 * R, 3000
    h = 2 * L / N
    g = (np.arange(N) + 0.5) * h - L
    X, Y = np.meshgrid(g, g)
    img = oracle.sersic(X.ravel(), Y.ravel(), [R, n, e1, e2, 0.0, 0.0, I0])
    # add the analytic tail beyond the box is negligible for these n at 12 R_eff? bound it
    flux = img.sum() * h * h
    assert flux == pytest.approx(expect, rel=3e-3)


def test_sersic_position_angle_sense():
    """e2 > 0 (phi = 45 deg) elongates the light along x = y."""
    l = [0.5, 1.5, 0.0, 0.3, 0.0, 0.0, 10.0]
    d = 0.4 / math.sqrt(2)
    on = oracle.sersic([d], [d], l)[0]
    off = oracle.sersic([-d], [d], l)[0]
    assert on > 1.5 * off
    l2 = [0.5, 1.5, 0.3, 0.0, 0.0, 0.0, 10.0]  # phi = 0: major axis along x
    assert oracle.sersic([0.4], [0.0], l2)[0] > 1.5 * oracle.sersic([0.0], [0.4], l2)[0]


@pytest.mark.parametrize("psi", [0.4, -1.1])
def test_sersic_rotation_covariance(psi):
    l = [0.6, 2.3, 0.11, -0.17, 0.03, -0.05, 50.0]
    x = RNG.uniform(-1.5, 1.5, 30)
    y = RNG.uniform(-1.5, 1.5, 30)
    a = oracle.sersic(x, y, l)
    e = complex(l[2], l[3]) * complex(math.cos(2 * psi), math.sin(2 * psi))
    xc, yc = _rot(l[4], l[5], psi)
    xr, yr = _rot(x, y, psi)
    b = oracle.sersic(xr, yr, [l[0], l[1], e.real, e.imag, xc, yc, l[6]])
    np.testing.assert_allclose(b, a, rtol=1e-12)


# ---------------------------------------------------- lens equation ---------

def test_ray_trace_is_lens_equation_and_source_is_conserved():
    """beta = theta - alpha_epl - alpha_ext, and the image-plane brightness is the
    source brightness at beta plus the lens light at theta."""
    p = inputs.draw_truth(np.random.default_rng(7))
    x = RNG.uniform(-2, 2, 50)
    y = RNG.uniform(-2, 2, 50)
    bx, by = oracle.ray_trace(x, y, p)
    ax, ay = oracle.epl_deflection(x, y, p[0:6])
    sx, sy = oracle.shear_deflection(x, y, p[6], p[7])
    np.testing.assert_allclose(bx, x - ax - sx, atol=1e-14)
    np.testing.assert_allclose(by, y - ay - sy, atol=1e-14)
    sb = oracle.surface_brightness(x, y, p)
    np.testing.assert_allclose(sb, oracle.sersic(bx, by, p[15:22]) + oracle.sersic(x, y, p[8:15]), rtol=1e-13)


# -------------------------------------------------- grid and binning --------

def _light_only(R=0.3, n=1.0, e1=0.0, e2=0.0, x=0.0, y=0.0, I0=10.0):
    """Parameter vector whose image is the lens light alone (source amplitude 0)."""
    p = np.zeros(22)
    p[0], p[1] = 1.0, 2.0
    p[8:15] = [R, n, e1, e2, x, y, I0]
    p[15:22] = [0.1, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    return p


def test_binning_is_mean_of_finer_grid():
    """The k-supersampled, averaged image equals the k x k block means of the
    k-times finer image at pixel scale / k: this pins the subpixel centres and the
    averaging of Sec. 2.1.1."""
    p = inputs.draw_truth(np.random.default_rng(3))
    H, W, k, d = 9, 12, 3, 0.065
    coarse = oracle.binned_image(p, H, W, k, d)
    fine = oracle.binned_image(p, k * H, k * W, 1, d / k)
    np.testing.assert_allclose(coarse, fine.reshape(H, k, W, k).mean(axis=(1, 3)), rtol=1e-13)


def test_grid_orientation_and_centre():
    """x grows with the column index and y with the row index; pixel centres are
    symmetric about (0, 0)."""
    H = W = 21
    d = 0.065
    img = oracle.binned_image(_light_only(R=0.1, x=0.0, y=0.0), H, W, 1, d)
    assert np.unravel_index(np.argmax(img), img.shape) == (10, 10)
    np.testing.assert_allclose(img, img[::-1, :], rtol=1e-13)
    np.testing.assert_allclose(img, img.T, rtol=1e-13)
    img = oracle.binned_image(_light_only(R=0.1, x=2 * d, y=0.0), H, W, 1, d)
    assert np.unravel_index(np.argmax(img), img.shape) == (10, 12)
    img = oracle.binned_image(_light_only(R=0.1, x=0.0, y=3 * d), H, W, 1, d)
    assert np.unravel_index(np.argmax(img), img.shape) == (13, 10)
    # even sizes: no pixel at the origin, image symmetric
    img = oracle.binned_image(_light_only(R=0.1), 10, 10, 2, d)
    np.testing.assert_allclose(img, img[::-1, ::-1], rtol=1e-13)


def test_binned_flux_matches_sersic_total():
    """Sum of pixel values x pixel area -> Sersic total flux (k = 4)."""
    R, n, I0, d = 0.2, 1.0, 1.0, 0.065
    bn = 1.9992 * n - 0.3271
    expect = 2 * math.pi * n * R * R * I0 * math.exp(bn) * math.gamma(2 * n) / bn ** (2 * n)
    img = oracle.binned_image(_light_only(R=R, n=n, I0=I0, e1=0.1), 81, 81, 4, d)
    assert img.sum() * d * d == pytest.approx(expect, rel=2e-3)


# ------------------------------------------------------- convolution --------

def test_convolution_delta_psf_is_identity():
    img = RNG.normal(size=(13, 17))
    delta = np.zeros((5, 5))
    delta[2, 2] = 1.0
    np.testing.assert_array_equal(oracle.convolve(img, delta), img)
    np.testing.assert_array_equal(oracle.convolve(img, np.ones((1, 1))), img)


@pytest.mark.parametrize("K", [1, 3, 5, 11])
def test_convolution_matches_scipy_same(K):
    """True convolution, zero padding, 'same' output: scipy.signal.convolve2d with an
    asymmetric kernel pins the flip direction."""
    img = RNG.normal(size=(16, 13))
    psf = RNG.uniform(0, 1, (K, K))
    np.testing.assert_allclose(oracle.convolve(img, psf), signal.convolve2d(img, psf, mode="same"), atol=1e-13)


def test_convolution_conserves_flux_inside():
    img = np.zeros((31, 31))
    img[12:19, 11:20] = RNG.uniform(0, 1, (7, 9))
    psf = inputs.gaussian_psf(11)
    assert oracle.convolve(img, psf).sum() == pytest.approx(img.sum(), rel=1e-12)


# -------------------------------------------------------- likelihood --------

def test_likelihood_zero_residual():
    M = RNG.uniform(0, 5, (8, 9))
    sig = RNG.uniform(0.01, 0.1, (8, 9))
    ll, c2 = oracle.likelihood_image(M, M, sig, 1000.0)
    assert c2 == 0.0
    v = sig ** 2 + M / 1000.0
    assert ll == pytest.approx(-0.5 * np.sum(np.log(2 * np.pi * v)), rel=1e-14)


def test_likelihood_gaussian_logpdf():
    """Without the Poisson term the likelihood is the product of normal densities;
    with it, each pixel is normal with variance sigma^2 + M/(G t_exp)."""
    M = RNG.uniform(0, 5, (8, 9))
    D = M + RNG.normal(0, 0.05, M.shape)
    sig = RNG.uniform(0.01, 0.1, M.shape)
    ll, c2 = oracle.likelihood_image(M, D, sig, 0.0)
    assert ll == pytest.approx(np.sum(stats.norm.logpdf(D, M, sig)), rel=1e-13)
    assert c2 == pytest.approx(np.sum(((D - M) / sig) ** 2), rel=1e-13)
    ll, _ = oracle.likelihood_image(M, D, sig, 250.0)
    assert ll == pytest.approx(np.sum(stats.norm.logpdf(D, M, np.sqrt(sig ** 2 + M / 250.0))), rel=1e-13)


def test_likelihood_variance_matches_poisson_noise():
    """Sec. 2.1.2: counts are Poisson with mean G t_exp M, so data drawn as
    Poisson(G t M)/(G t) + N(0, sigma^2) has E[chi^2] = number of pixels."""
    rng = np.random.default_rng(99)
    M = rng.uniform(1.0, 50.0, (200, 200))
    gt, sig = 20.0, 0.05
    D = inputs.add_noise(rng, M, sig, gt)
    _, c2 = oracle.likelihood_image(M, D, sig, gt)
    n = M.size
    assert abs(c2 / n - 1.0) < 5 * math.sqrt(2.0 / n)
    # a variance off by the gain would be far outside that band
    _, c2_wrong = oracle.likelihood_image(M, D, sig, gt * 2.0)
    assert abs(c2_wrong / n - 1.0) > 20 * math.sqrt(2.0 / n)


# ------------------------------------------------------------- whole chain --

def _small_system(seed=0, H=14, W=14, k=2, K=5, gain=1000.0):
    rng = np.random.default_rng(seed)
    truth = inputs.draw_truth(rng)
    psf = inputs.moffat_psf(K)
    model = oracle.simulate(truth, H, W, psf, 0.065, k)[0]
    D = inputs.add_noise(rng, model, 0.01, gain)
    return truth, D, psf


def test_simulate_is_binning_then_area_then_convolution():
    truth, _, psf = _small_system()
    pre = oracle.binned_image(truth, 14, 14, 2, 0.065)
    np.testing.assert_allclose(oracle.simulate(truth, 14, 14, psf, 0.065, 2)[0],
                               oracle.convolve(pre * 0.065 ** 2, psf), rtol=1e-14)


def test_simulated_pixels_sum_to_the_total_flux():
    """A pixel records the flux falling on it: with a delta PSF the pixel values
    of a simulated light-only image sum to the Sersic total flux
    2 pi n R^2 I0 e^{b_n} Gamma(2n) / b_n^{2n} (counts/s), for two pixel scales."""
    R, n, I0 = 0.2, 1.5, 3.0
    bn = 1.9992 * n - 0.3271
    expect = 2 * math.pi * n * R * R * I0 * math.exp(bn) * math.gamma(2 * n) / bn ** (2 * n)
    delta = np.zeros((1, 1))
    delta[0, 0] = 1.0
    for d, H in ((0.065, 81), (0.03, 161)):
        img = oracle.simulate(_light_only(R=R, n=n, I0=I0, e1=0.1), H, H, delta, d, 4)[0]
        assert img.sum() == pytest.approx(expect, rel=3e-3)


def test_whole_model_rot90_covariance():
    """np.rot90 of the image array maps pixel (x, y) to (-y, x) under x = column,
    y = row. Transforming every centre c -> (y_c, -x_c), every ellipticity and the
    shear by e^{-i pi} = -1 and rotating the (asymmetric) PSF the same way must
    give the rotated image: pins grid orientation, rotation senses and the
    convolution together."""
    rng = np.random.default_rng(5)
    p = inputs.draw_truth(rng)
    psf = RNG.uniform(0, 1, (5, 5))
    a = oracle.simulate(p, 16, 16, psf, 0.065, 2)[0]
    q = p.copy()
    for ix, iy in ((4, 5), (12, 13), (19, 20)):
        q[ix], q[iy] = p[iy], -p[ix]
    for j in (2, 3, 6, 7, 10, 11, 17, 18):
        q[j] = -p[j]
    b = oracle.simulate(q, 16, 16, np.rot90(psf), 0.065, 2)[0]
    np.testing.assert_allclose(b, np.rot90(a), rtol=1e-11, atol=1e-12)


def test_whole_model_transpose_covariance():
    """Reflection across x = y: centres swap, e1 and gamma_ext1 flip sign."""
    p = inputs.draw_truth(np.random.default_rng(6))
    psf = RNG.uniform(0, 1, (3, 3))
    a = oracle.simulate(p, 12, 12, psf, 0.065, 3)[0]
    q = p.copy()
    for ix, iy in ((4, 5), (12, 13), (19, 20)):
        q[ix], q[iy] = p[iy], p[ix]
    for j in (2, 6, 10, 17):
        q[j] = -p[j]
    b = oracle.simulate(q, 12, 12, psf.T, 0.065, 3)[0]
    np.testing.assert_allclose(b, a.T, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    """Forward-mode dual gradient of log L vs central finite differences with a
    Richardson step (h and h/2)."""
    truth, D, psf = _small_system(seed)
    rng = np.random.default_rng(100 + seed)
    p = inputs.draw_perturbed(rng, truth, 1)[0]
    sig = np.full(D.shape, 0.01)
    ll, _, g = oracle.loglik(p, D, sig, psf, 0.065, 2, 1000.0, grad=True)
    fd = np.empty(22)
    for i in range(22):
        h = 1e-4 * max(1.0, abs(p[i]))

        def cd(hh):
            pp, pm = p.copy(), p.copy()
            pp[i] += hh
            pm[i] -= hh
            lp = oracle.loglik(pp, D, sig, psf, 0.065, 2, 1000.0)[0][0]
            lm = oracle.loglik(pm, D, sig, psf, 0.065, 2, 1000.0)[0][0]
            return (lp - lm) / (2 * hh)

        fd[i] = (4 * cd(h / 2) - cd(h)) / 3
    scale = np.abs(g) + 1e-6 * np.max(np.abs(g))
    assert np.max(np.abs(g[0] - fd) / scale) < 1e-5
    assert np.isfinite(ll).all()


def test_loglik_value_path_equals_gradient_path():
    truth, D, psf = _small_system(4)
    ps = inputs.draw_perturbed(np.random.default_rng(4), truth, 5)
    a = oracle.loglik(ps, D, 0.01, psf, 0.065, 2, 1000.0)
    b = oracle.loglik(ps, D, 0.01, psf, 0.065, 2, 1000.0, grad=True)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-13)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-13)
    model = oracle.simulate(ps, 14, 14, psf, 0.065, 2)
    for i in range(5):
        ll, c2 = oracle.likelihood_image(model[i], D, 0.01, 1000.0)
        assert a[0][i] == pytest.approx(ll, rel=1e-13)
        assert a[1][i] == pytest.approx(c2, rel=1e-13)


def test_model_jacobian_matches_differences_and_gradient():
    """dM/dparams from the oracle's duals: central differences of the model, and
    the chain rule J^T dlogL/dM reproduces the log L gradient."""
    truth, D, psf = _small_system(8, H=10, W=12, k=2, K=3)
    p = inputs.draw_perturbed(np.random.default_rng(8), truth, 1)[0]
    M, J = oracle.model_jacobian(p, 10, 12, psf, 0.065, 2)
    np.testing.assert_allclose(M, oracle.simulate(p, 10, 12, psf, 0.065, 2)[0], rtol=1e-14)
    def cd(i, h):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        return (oracle.simulate(pp, 10, 12, psf, 0.065, 2)[0] - oracle.simulate(pm, 10, 12, psf, 0.065, 2)[0]) / (2 * h)

    for i in (0, 1, 3, 9, 16, 19):
        h = 1e-4 * max(1.0, abs(p[i]))
        fd = (4 * cd(i, h / 2) - cd(i, h)) / 3
        np.testing.assert_allclose(J[:, :, i], fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    G, sig = 1000.0, 0.01
    v = sig ** 2 + M / G
    r = D - M
    gpix = r / v + (r * r / (v * v) - 1 / v) / (2 * G)
    _, _, g = oracle.loglik(p, D, sig, psf, 0.065, 2, G, grad=True)
    np.testing.assert_allclose(np.einsum("hw,hwj->j", gpix, J), g[0], rtol=1e-9, atol=1e-9 * np.abs(g).max())
