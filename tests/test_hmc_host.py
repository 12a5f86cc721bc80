"""Host logic of the HMC driver: dual-averaging step-size adaptation
(Hoffman & Gelman 2014) on a synthetic acceptance curve a(eps) = exp(-eps),
whose target-0.75 step size is -log 0.75 in closed form."""
import math

import pytest

pytest.importorskip("torch")

from paper_2202_07663_gb300 import hmc  # noqa: E402


def test_dual_averaging_converges_to_target_step_size():
    da = hmc.DualAveraging(1.0, target=0.75)
    eps = 1.0
    for _ in range(2000):
        eps = da.update(math.exp(-eps))
    assert abs(da.final() - (-math.log(0.75))) < 0.01 * -math.log(0.75)


def test_dual_averaging_moves_the_right_way():
    # acceptance too low -> smaller steps; too high -> larger steps
    lo = hmc.DualAveraging(0.1, target=0.75)
    hi = hmc.DualAveraging(0.1, target=0.75)
    assert lo.update(0.1) < 1.0 and hi.update(1.0) > lo.update(0.1)
    # the first proposal sits at mu = log(10 eps0) shrunk by the error
    d = hmc.DualAveraging(0.2, target=0.75)
    e1 = d.update(0.75)
    assert abs(e1 - 2.0) < 1e-12
