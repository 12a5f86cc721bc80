"""Continuous batching on the GPU: the graph-replayed batcher against single
calls, each request's result alone vs in a mixed stream (within the parity
tolerance), the arena budget error, and a short real-time stream."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402
from gpu_common import assert_plain_parity, assert_sum_order_close  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import build
    build.build()
    oracle.build()
    from paper_2202_07663_gb300 import abi, serving
    return abi, serving


def _stream(n, rate, seed):
    return inputs.serving_stream(n=n, rate_hz=rate, seed=seed, bmin=64, bmax=700)


def test_batcher_matches_single_calls(mods):
    abi, serving = mods
    dev = torch.device("cuda")
    specs = [inputs.SystemSpec(60, 60, 2, 11), inputs.SystemSpec(80, 80, 4, 21), inputs.SystemSpec(40, 40, 2, 5),
             inputs.SystemSpec(120, 120, 2, 21)]
    reqs = serving.make_requests([inputs.LensRequest(i, 0.0, sp, 100 + 37 * i, 900 + i) for i, sp in enumerate(specs)],
                                 dev)
    b = abi.Batcher(16, 512 << 20, 128, 128, 21)
    systems, ps, outs = [], [], []
    for r in reqs:
        s = abi.GLSystem(r.image, r.psf, r.spec.pixel_scale, r.spec.k, r.spec.gain_exposure, sigma_bkg=r.spec.sigma_bkg)
        p = torch.from_numpy(r.params).to(dev)
        systems.append(s)
        ps.append(p)
        outs.append((torch.empty(p.shape[0], dtype=torch.float64, device=dev),
                     torch.empty(p.shape[0], 22, dtype=torch.float64, device=dev)))
    for _ in range(2):  # two replays of the same graph
        b.run(systems, [p.data_ptr() for p in ps], [p.shape[0] for p in ps], [o[0].data_ptr() for o in outs],
              [o[1].data_ptr() for o in outs])
    torch.cuda.synchronize()
    for s, p, (ll, g) in zip(systems, ps, outs):
        rl, rg = s.loglik_grad(p)
        # gradients are the same bits; the batcher's convolution blocks (sized
        # for its largest image) and a single call's sum log L in other orders
        assert_sum_order_close(ll.cpu().numpy(), rl.cpu().numpy(), "batcher vs single")
        np.testing.assert_array_equal(g.cpu().numpy(), rg.cpu().numpy())
    # a batch whose scratch exceeds the arena is refused
    small = abi.Batcher(4, 1 << 20, 128, 128, 21)
    with pytest.raises(abi.GLError) as ei:
        small.run(systems[:1], [ps[0].data_ptr()], [ps[0].shape[0]], [outs[0][0].data_ptr()], [outs[0][1].data_ptr()])
    assert ei.value.code == -5
    for s in systems:
        s.close()
    b.close()
    small.close()


def test_single_segment_batch_is_the_single_call(mods):
    """A batch of one segment takes the launch sequence of a single-system
    call (on the batcher's arena): the same bits as gl_loglik_grad, twice in
    a row, and on a second stream after the first."""
    abi, serving = mods
    dev = torch.device("cuda")
    reqs = serving.make_requests([inputs.LensRequest(0, 0.0, inputs.SystemSpec(80, 80, 2, 11), 50, 901),
                                  inputs.LensRequest(1, 0.0, inputs.SystemSpec(100, 100, 4, 21), 300, 902)], dev)
    b = abi.Batcher(8, 256 << 20, 128, 128, 21)
    other = torch.cuda.Stream()
    for r in reqs:
        s = abi.GLSystem(r.image, r.psf, r.spec.pixel_scale, r.spec.k, r.spec.gain_exposure, sigma_bkg=r.spec.sigma_bkg)
        p = torch.from_numpy(r.params).to(dev)
        rl, rg = [t.cpu().numpy() for t in s.loglik_grad(p)]
        for stream in (None, None, other.cuda_stream):
            ll = torch.full((p.shape[0],), float("nan"), dtype=torch.float64, device=dev)
            g = torch.full((p.shape[0], 22), float("nan"), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            b.run([s], [p.data_ptr()], [p.shape[0]], [ll.data_ptr()], [g.data_ptr()], stream=stream)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(ll.cpu().numpy(), rl)
            np.testing.assert_array_equal(g.cpu().numpy(), rg)
        s.close()
    b.close()


def test_each_result_is_the_same_alone_and_in_the_mix(mods):
    abi, serving = mods
    dev = torch.device("cuda")
    reqs = serving.make_requests(_stream(8, 200.0, 77), dev)
    srv = serving.LensServer(budget_bytes=1 << 30, arena_bytes=256 << 20, max_segments=6, chunk=200,
                             max_H=128, max_W=128, max_K=21)
    stats, res = srv.serve(reqs, realtime=False, keep_results=True)
    srv.close()
    assert stats.n == len(reqs) and stats.batches > len(reqs) // 6
    for r in reqs:
        s = abi.GLSystem(r.image, r.psf, r.spec.pixel_scale, r.spec.k, r.spec.gain_exposure, sigma_bkg=r.spec.sigma_bkg)
        ll, g = s.loglik_grad(torch.from_numpy(r.params).to(dev))
        s.close()
        ll, g = ll.cpu().numpy(), g.cpu().numpy()
        mix_ll, mix_g = res[r.index]
        assert_plain_parity(mix_ll, mix_g, ll, g, "request %d alone vs in the mix" % r.index)
        # the differences are the grouping of rays into tiles and, for requests of
        # fewer vectors than SMs served alone, the order of the FP32 log-L sums:
        # rounding of pixel terms whose scale the largest |log L| bounds
        assert np.max(np.abs(mix_ll - ll)) < 1e-6 * np.max(np.abs(ll))


def test_realtime_stream(mods):
    abi, serving = mods
    dev = torch.device("cuda")
    reqs = serving.make_requests(_stream(40, 200.0, 78), dev)
    srv = serving.LensServer(budget_bytes=1 << 30, arena_bytes=512 << 20, max_segments=16, chunk=1024)
    stats, _ = srv.serve(reqs, realtime=True)
    srv.close()
    summ = stats.summary()
    assert summ["lenses"] == 40
    assert 0 < summ["latency_ms"]["p50"] <= summ["latency_ms"]["p99"] < 5000
    base = serving.serve_one_call_per_lens(reqs, realtime=False)
    assert base.n == 40 and np.all(base.latencies_s > 0)
