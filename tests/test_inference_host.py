"""Host-side pieces of the inference layer, on CPU:

- the variational parameters' packing (``vi.pack``/``vi.unpack``) has the
  layout of the oracle's Cholesky bijector (mean, then the lower triangle row
  by row with the log of the diagonal) and round-trips;
- the VI learning-rate schedule is the oracle's Table 1 schedule;
- ``pipeline.model_system`` refuses a bad preconditioner and fewer starts,
  draws or chains than processes before it touches the GPU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import vi_oracle as vo  # noqa: E402


def test_vi_packing_matches_the_oracle_layout():
    from paper_2202_07663_gb300 import vi
    rng = np.random.default_rng(3)
    for d in (1, 2, 7, 22):
        mu = rng.normal(size=d)
        L = np.tril(rng.normal(size=(d, d)), -1) + np.diag(np.exp(rng.normal(size=d)))
        phi = vi.pack(torch.from_numpy(mu), torch.from_numpy(L))
        assert phi.shape == (vi.n_params(d),) and vi.n_params(d) == vo.n_params(d)
        np.testing.assert_allclose(phi.numpy(), vo.pack(mu, L), rtol=0, atol=1e-15)
        mu2, L2 = vi.unpack(phi, d)
        np.testing.assert_allclose(mu2.numpy(), mu, rtol=0, atol=0)
        np.testing.assert_allclose(L2.numpy(), L, rtol=1e-15, atol=0)
        mu3, L3 = vo.unpack(phi.numpy(), d)
        np.testing.assert_allclose(L2.numpy(), L3, rtol=1e-15, atol=0)


def test_vi_schedule_is_table_1():
    from paper_2202_07663_gb300 import vi
    for t in (0, 1, 100, 250, 499, 500, 501, 999):
        assert vi.quadratic_warmup(t) == pytest.approx(vo.learning_rate(t), rel=0, abs=1e-18)
    assert vi.quadratic_warmup(0) == 0.0 and vi.quadratic_warmup(10_000) == pytest.approx(vo.LR_PEAK)
    assert vi.quadratic_warmup(250) == pytest.approx(vo.LR_PEAK * (1 - 0.25))


def test_pipeline_argument_checks_come_first():
    from paper_2202_07663_gb300 import pipeline
    starts = torch.zeros(4, 22)
    with pytest.raises(ValueError, match="preconditioner"):
        pipeline.model_system(object(), starts, preconditioner="diag")


def test_pipeline_needs_a_unit_per_process(monkeypatch):
    from paper_2202_07663_gb300 import distributed, pipeline
    monkeypatch.setattr(distributed, "world", lambda group=None: (0, 8))
    with pytest.raises(ValueError, match="fewer starts"):
        pipeline.model_system(object(), torch.zeros(4, 22), group=object())
    with pytest.raises(ValueError, match="fewer starts"):
        pipeline.model_system(object(), torch.zeros(16, 22), chains=5, group=object())
