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


def test_jitter_sequence_matches_the_oracle():
    from oracle import hmc_oracle as ho
    assert [hmc.van_der_corput(m) for m in range(1, 200)] == [ho.van_der_corput(m) for m in range(1, 200)]


def test_trajectory_adam_climbs_a_chees_curve():
    # ChEES(T) = d sin^2 T (standard normal, exact flow): gradient in log T is
    # T d sin 2T; the ascent settles at the quarter period pi/2
    ta = hmc.TrajectoryAdam(0.3)
    T = 0.3
    for _ in range(3000):
        T = ta.update(T * 22 * math.sin(2 * T))
    assert abs(T - math.pi / 2) < 0.05
    # capped, and a non-finite gradient leaves T alone
    tb = hmc.TrajectoryAdam(1.0, t_max=1.2)
    for _ in range(100):
        Tb = tb.update(5.0)
    assert Tb == pytest.approx(1.2)
    assert tb.update(float("nan")) == pytest.approx(1.2)
