"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU: one JSON line with the benchmark's keys, the oracle's own
rate in ``value``, ``cpu_baseline`` and ``e2e``, no host-device bytes and at
least three warm-up steps; ranks other than 0 print nothing and exit 0.
The clocks record of the benchmark line is parsed from nvidia-smi samples,
and the EPL series length behind its flop count follows its stated rule."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    pytest.importorskip("numpy")
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    # fewer than three warm-up steps are raised to three, as for the GPU arm
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_summary_parses_throttle_reasons():
    """The clocks record of the benchmark line: median SM clock under load,
    the maximum clock, and which throttle reasons were active at any sample."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.lines = ["0, 2070, 2070, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "0, 2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = ["0, 1500, 2070, 700.0, 0x0000000000000048, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary() is None


def test_series_terms_by_brute_force():
    """The per-vector EPL series length behind the roofline's flop count:
    the smallest N with |a_(N+1)| f^(N+1) / (1 - f max(1, c_(N+2))) <= tol,
    a_n = c_1 ... c_n, c_k = (2k - 2 + t) / (2k + 2 - t), t = gamma - 1,
    f = |e| (at least one term in the adjoint), by a plain loop."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench

    def brute(gamma, e1, e2, adjoint):
        f, t = math.hypot(e1, e2), gamma - 1.0
        c = lambda k: (2 * k - 2 + t) / (2 * k + 2 - t)   # noqa: E731
        a = 1.0
        for N in range(0, bench.NMAX + 1):
            a *= c(N + 1)                                  # a_(N+1)
            r = min(f * max(1.0, c(N + 2)), 0.999999)
            if abs(a) * f ** (N + 1) / (1.0 - r) <= bench.SERIES_TOL:
                return max(N, 1) if adjoint else N
        return max(bench.NMAX, 1) if adjoint else bench.NMAX

    rng = np.random.default_rng(9)
    P = np.zeros((400, 22))
    P[:, 1] = rng.uniform(1.5, 2.5, 400)
    P[:, 2:4] = rng.normal(0.0, 0.15, (400, 2))
    P[:4, 2:4] = 0.0                          # circular: no series term needed
    P[4:8, 2] = [0.5, 0.7, 0.9, 0.95]         # long series
    for adjoint in (False, True):
        N = bench.series_terms(P, adjoint)
        ref = [brute(P[i, 1], P[i, 2], P[i, 3], adjoint) for i in range(len(P))]
        assert list(N) == ref
    assert list(bench.series_terms(P[:4], False)) == [0] * 4 and list(bench.series_terms(P[:4], True)) == [1] * 4
