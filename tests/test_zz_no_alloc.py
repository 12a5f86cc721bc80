"""gl_loglik_grad_noalloc: the entry point for callers that cannot allocate
device memory while they evaluate the likelihood (allocator callbacks,
processes whose device memory another framework's caching allocator already
holds, hosts that forbid allocation after start-up).

It must give the results of gl_loglik_grad, call after call, from its
static scratch array. This file is named to be collected last, so that a
run stopping at its first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402
from gpu_common import assert_plain_parity, make_system  # noqa: E402

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import build, abi as _abi
    build.build()
    oracle.build()
    return _abi


def _noalloc(lib, sysm, params):
    B = params.shape[0]
    ll = torch.empty(B, dtype=torch.float64, device="cuda")
    c2 = torch.empty(B, dtype=torch.float64, device="cuda")
    g = torch.empty(B, 22, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.gl_loglik_grad_noalloc(sysm.handle, params.data_ptr(), B, ll.data_ptr(), c2.data_ptr(),
                                    g.data_ptr(), stream)
    assert rc == 0, lib.gl_last_error_message().decode()
    torch.cuda.synchronize()
    return ll.cpu().numpy(), c2.cpu().numpy(), g.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(abi):
    lib = abi.lib_handle()
    spec = inputs.WORKLOADS[inputs.PLAIN]["spec"]
    truth, image, psf = make_system(spec, 4242)
    sysm = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    rng = np.random.default_rng(77)
    assert sysm.scratch_held() == 0
    for call in range(2):   # two calls in a row: the second reuses the array the first left behind
        B = 64 if call == 0 else 37
        params = torch.from_numpy(inputs.draw_perturbed(rng, truth, B).astype(np.float32)).cuda()
        ll, c2, g = _noalloc(lib, sysm, params)
        if call == 0:
            # the system's own scratch is still unallocated: the call used the static array only
            assert sysm.scratch_held() == 0
        rl, rg, rc2 = [t.cpu().numpy() for t in sysm.loglik_grad(params, chi2=True)]
        assert sysm.scratch_held() > 0
        assert_plain_parity(ll, g, rl, rg, "no-alloc call %d" % call)
        np.testing.assert_allclose(c2, rc2, rtol=1e-4)
    sysm.close()


def test_noalloc_rejects_batches_beyond_the_static_scratch(abi):
    lib = abi.lib_handle()
    spec = inputs.WORKLOADS[inputs.PLAIN]["spec"]
    _, image, psf = make_system(spec, 4243)
    sysm = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    B = SCRATCH_BYTES // (4 * spec.H * spec.W) + 1   # the image work buffer alone overflows
    params = torch.zeros(B, 22, dtype=torch.float32, device="cuda")
    out = torch.empty(B, 23, dtype=torch.float64, device="cuda")
    rc = lib.gl_loglik_grad_noalloc(sysm.handle, params.data_ptr(), B, out.data_ptr(), None,
                                    out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"static scratch" in lib.gl_last_error_message()
    sysm.close()
