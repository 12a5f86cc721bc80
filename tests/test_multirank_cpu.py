"""World-size-2 gloo run of the benchmark's multi-rank host logic on CPU:
per-rank batches differ, the step time is the max over ranks, and the
whole-job rate counts every rank's vectors (weak scaling, no data-path
collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import bench
    from paper_2202_07663_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.rank_param_seed(bench.WORKLOAD, rank)
        p = inputs.draw_box(np.random.default_rng(seed), 8)
        t = 1.0 + rank  # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, torch.device("cpu"), world)
        out[rank] = (seed, float(p[0, 0]), tmax, bench.whole_job_rate(world, 4096, tmax))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] != res[1][0] and res[0][1] != res[1][1]   # distinct batches per rank
    assert res[0][2] == res[1][2] == 2.0                        # max over ranks
    assert res[0][3] == pytest.approx(2 * 4096 / 2.0)           # all ranks' vectors / slowest time
