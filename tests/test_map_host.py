"""The product's prior (passed to the MAP kernels) and the oracle's prior are
two transcriptions of Eq. sim-dist (prior column); they must agree."""
import pytest

pytest.importorskip("torch")


def test_product_and_oracle_priors_agree():
    from oracle import map_oracle as mo
    from paper_2202_07663_gb300 import abi, map as gmap
    names = {abi.GL_PRIOR_NORMAL: "normal", abi.GL_PRIOR_LOGNORMAL: "lognormal",
             abi.GL_PRIOR_TRUNCNORMAL: "truncnormal", abi.GL_PRIOR_UNIFORM: "uniform"}
    for mine, ref in zip(gmap.PAPER_PRIOR, mo.PRIOR):
        kind, a, b, c, d = mine
        assert names[kind] == ref[0]
        nparam = len(ref) - 1
        assert (a, b, c, d)[:nparam] == tuple(ref[1:])


def test_linear_schedule():
    from paper_2202_07663_gb300 import map as gmap
    assert gmap.linear_lr(0) == 1e-2
    assert gmap.linear_lr(300) == pytest.approx(1e-3)
    assert gmap.linear_lr(10_000) == pytest.approx(1e-3)
