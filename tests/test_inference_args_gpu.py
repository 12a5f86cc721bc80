"""Argument checking of the inference-layer entry points: every bad call
returns GL_ERR_INVALID_ARG (-1) before launching anything, and B = 0 is a
no-op where the header says so."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

INVALID = -1


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import abi, build
    build.build()
    return abi.lib_handle()


def _buf(n, dtype=torch.float64):
    return torch.zeros(max(n, 1), dtype=dtype, device="cuda")


def test_hmc_entry_points(lib):
    st = torch.cuda.current_stream().cuda_stream
    q, p, g, im = _buf(44), _buf(44), _buf(44), _buf(22)
    assert lib.gl_hmc_leapfrog(2, 22, q.data_ptr(), p.data_ptr(), g.data_ptr(), im.data_ptr(), 0.1, 1.0, None, st) == 0
    assert lib.gl_hmc_leapfrog(2, 0, q.data_ptr(), p.data_ptr(), g.data_ptr(), im.data_ptr(), 0.1, 1.0, None,
                               st) == INVALID
    assert lib.gl_hmc_leapfrog(2, 22, None, p.data_ptr(), g.data_ptr(), im.data_ptr(), 0.1, 1.0, None, st) == INVALID
    assert lib.gl_hmc_leapfrog(2, 22, q.data_ptr(), p.data_ptr(), g.data_ptr(), im.data_ptr(), float("nan"), 1.0,
                               None, st) == INVALID
    assert lib.gl_hmc_leapfrog_dev(2, 22, q.data_ptr(), p.data_ptr(), g.data_ptr(), im.data_ptr(), None, 1.0, None,
                                   st) == INVALID
    assert lib.gl_hmc_leapfrog(0, 22, None, None, None, None, 0.1, 1.0, None, st) == 0
    out = _buf(3)
    assert lib.gl_hmc_chees(0, 22, q.data_ptr(), q.data_ptr(), p.data_ptr(), im.data_ptr(), out.data_ptr(), 1.0,
                            out.data_ptr(), st) == INVALID
    assert lib.gl_hmc_chees(2, 2000, q.data_ptr(), q.data_ptr(), p.data_ptr(), im.data_ptr(), out.data_ptr(), 1.0,
                            out.data_ptr(), st) == INVALID
    assert lib.gl_hmc_chees(2, 22, q.data_ptr(), q.data_ptr(), None, im.data_ptr(), out.data_ptr(), 1.0,
                            out.data_ptr(), st) == INVALID
    L, mu, z = _buf(22 * 22), _buf(22), _buf(44)
    assert lib.gl_hmc_affine(2, 65, q.data_ptr(), mu.data_ptr(), L.data_ptr(), z.data_ptr(), None, st) == INVALID
    assert lib.gl_hmc_affine(2, 22, q.data_ptr(), mu.data_ptr(), L.data_ptr(), q.data_ptr(), None, st) == INVALID
    assert lib.gl_hmc_affine_pullback(2, 22, q.data_ptr(), L.data_ptr(), q.data_ptr(), st) == INVALID
    torch.cuda.synchronize()


def test_vi_and_posterior_entry_points(lib):
    from paper_2202_07663_gb300 import map as gmap
    st = torch.cuda.current_stream().cuda_stream
    assert lib.gl_vi_param_count(22) == 22 + 253
    assert lib.gl_vi_param_count(0) == 0 and lib.gl_vi_param_count(33) == 0
    assert lib.gl_vi_workspace_bytes(0, 22) == 0
    n, d = 8, 22
    P = lib.gl_vi_param_count(d)
    eps, phi, z, lp, gz = _buf(n * d), _buf(P), _buf(n * d), _buf(n), _buf(n * d)
    g, loss = _buf(P), _buf(1)
    ws = torch.empty(lib.gl_vi_workspace_bytes(n, d), dtype=torch.uint8, device="cuda")
    pt = gmap.prior_table()
    assert lib.gl_vi_sample(n, 7, eps.data_ptr(), phi.data_ptr(), ctypes.addressof(pt), z.data_ptr(), None,
                            st) == INVALID   # a prior needs d = 22
    assert lib.gl_vi_sample(n, 40, eps.data_ptr(), phi.data_ptr(), None, z.data_ptr(), None, st) == INVALID
    args = (n, d, eps.data_ptr(), lp.data_ptr())
    assert lib.gl_vi_step(*args, None, 1, phi.data_ptr(), None, None, 0, 0.0, 0.9, 0.999, 1e-8, g.data_ptr(),
                          loss.data_ptr(), ws.data_ptr(), st) == INVALID   # pathwise needs grad_z
    assert lib.gl_vi_step(*args, gz.data_ptr(), 7, phi.data_ptr(), None, None, 0, 0.0, 0.9, 0.999, 1e-8,
                          g.data_ptr(), loss.data_ptr(), ws.data_ptr(), st) == INVALID   # unknown estimator
    assert lib.gl_vi_step(*args, gz.data_ptr(), 1, phi.data_ptr(), g.data_ptr(), None, 1, 1e-3, 0.9, 0.999, 1e-8,
                          g.data_ptr(), loss.data_ptr(), ws.data_ptr(), st) == INVALID   # m without v
    assert lib.gl_vi_step(*args, gz.data_ptr(), 1, phi.data_ptr(), None, None, 0, 0.0, 0.9, 0.999, 1e-8,
                          g.data_ptr(), loss.data_ptr(), None, st) == INVALID   # no workspace
    bad = gmap.prior_table()
    bad[0].b = -1.0
    assert lib.gl_posterior_grad(n, z.data_ptr(), lp.data_ptr(), None, ctypes.addressof(bad), lp.data_ptr(), None,
                                 st) == INVALID
    assert lib.gl_posterior_grad(n, z.data_ptr(), lp.data_ptr(), gz.data_ptr(), ctypes.addressof(pt),
                                 lp.data_ptr(), None, st) == INVALID   # gradient in but no gradient out
    torch.cuda.synchronize()
