"""gl_psf_factor (host only): the separable terms of a PSF that the
convolution stage uses instead of the K x K stencil.

Pinned against numpy's SVD, not against the library's own Jacobi sweeps:
the rank follows the stated rule (the fewest terms whose dropped singular
values have a root sum of squares of at most 2^-24 ||P||_F; 0 when 4 R > K),
the row factors carry the singular values, the column factors are
orthonormal, and the terms rebuild the PSF to FP32 rounding. A sampled
Gaussian is an outer product of two 1-D Gaussians (rank 1 exactly); a
Moffat profile is not separable.
"""
import numpy as np
import pytest

from paper_2202_07663_gb300 import inputs


@pytest.fixture(scope="module")
def abi():
    from paper_2202_07663_gb300 import build
    build.build()
    from paper_2202_07663_gb300 import abi as mod
    return mod


def _rank_rule(psf):
    s = np.linalg.svd(psf.astype(np.float64), compute_uv=False)
    total = np.sum(s * s)
    R = len(s)
    tail = 0.0
    while R > 1 and tail + s[R - 1] ** 2 <= 2.0 ** -48 * total:
        tail += s[R - 1] ** 2
        R -= 1
    return (R if 4 * R <= psf.shape[0] else 0), s


def _check_terms(psf, R, fac, s):
    K = psf.shape[0]
    assert fac.shape == (R, 2, K)
    u, v = fac[:, 0, :].astype(np.float64), fac[:, 1, :].astype(np.float64)
    np.testing.assert_allclose(v @ v.T, np.eye(R), atol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), s[:R], rtol=1e-5)
    rebuilt = np.einsum("ri,rj->ij", u, v)
    assert np.max(np.abs(rebuilt - psf)) <= 2e-7 * np.max(np.abs(psf))


@pytest.mark.parametrize("K", [5, 11, 21, 41])
def test_gaussian_psf_is_rank_one(abi, K):
    psf = inputs.gaussian_psf(K)
    R, fac = abi.psf_factor(psf)
    expect, s = _rank_rule(psf)
    assert R == expect == 1
    _check_terms(psf, R, fac, s)


def test_delta_and_zero_psfs(abi):
    """A delta PSF (the identity convolution) is rank 1 with unit factors;
    an all-zero PSF keeps the 2-D form (no norm to compare against)."""
    K = 11
    d = np.zeros((K, K), np.float32)
    d[5, 5] = 1.0
    R, fac = abi.psf_factor(d)
    assert R == 1
    np.testing.assert_allclose(np.outer(fac[0, 0], fac[0, 1]), d, atol=1e-7)
    assert abi.psf_factor(np.zeros((K, K), np.float32))[0] == 0


def test_sum_of_two_gaussians_is_rank_two(abi):
    x = np.arange(21) - 10.0
    g1, g2 = np.exp(-0.5 * (x / 1.3) ** 2), np.exp(-0.5 * ((x - 1.0) / 3.1) ** 2)
    psf = (np.outer(g1, g1) + 0.2 * np.outer(g2, g2[::-1])).astype(np.float32)
    psf /= psf.sum()
    R, fac = abi.psf_factor(psf)
    expect, s = _rank_rule(psf)
    assert R == expect == 2
    _check_terms(psf, R, fac, s)


@pytest.mark.parametrize("psf", [inputs.moffat_psf(21), inputs.moffat_psf(11),
                                 np.random.default_rng(3).uniform(size=(9, 9)).astype(np.float32),
                                 np.ones((1, 1), np.float32), np.ones((3, 3), np.float32)])
def test_kept_two_dimensional(abi, psf):
    """Moffat and random PSFs have too many terms; sides below 4 never pay
    for the 1-D passes (4 R > K even at R = 1)."""
    R, fac = abi.psf_factor(psf)
    assert R == 0 and fac.shape == (0, 2, psf.shape[0])
    assert _rank_rule(psf)[0] == 0


def test_bad_arguments(abi):
    lib = abi.lib_handle()
    import ctypes
    r = ctypes.c_int(-7)
    psf = np.ascontiguousarray(inputs.gaussian_psf(11), np.float32)
    assert lib.gl_psf_factor(psf.ctypes.data, 10, None, 0, ctypes.addressof(r)) == abi.GL_ERR_INVALID_ARG
    bad = psf.copy()
    bad[3, 4] = np.nan
    assert lib.gl_psf_factor(bad.ctypes.data, 11, None, 0, ctypes.addressof(r)) == abi.GL_ERR_INVALID_ARG
    out = np.zeros(21, np.float32)   # one term needs 2 K = 22 floats
    assert lib.gl_psf_factor(psf.ctypes.data, 11, out.ctypes.data, out.size, ctypes.addressof(r)) == \
        abi.GL_ERR_INVALID_ARG
    assert lib.gl_psf_factor(psf.ctypes.data, 11, None, 0, ctypes.addressof(r)) == abi.GL_OK and r.value == 1
