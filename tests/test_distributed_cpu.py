"""Host logic of inference spread over processes (``distributed``), run as
gloo ranks on CPU: row shards, rank-ordered gathers, the global best start,
and the global quantities the samplers adapt on (the mean acceptance
probability for dual averaging, the ChEES gradient on all chains), which
every rank must hold bit for bit, equal to a single process's."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_rows_in_rank_order():
    from paper_2202_07663_gb300 import distributed as D
    for n in (0, 1, 2, 5, 50, 300, 301):
        for size in (1, 2, 3, 4, 7):
            spans = [D.shard(n, r, size) for r in range(size)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(size - 1))
            c = D.counts(n, size)
            assert sum(c) == n and max(c) - min(c) <= 1 and c == sorted(c, reverse=True)
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def test_single_process_is_local():
    from paper_2202_07663_gb300 import distributed as D
    x = torch.arange(6.0).reshape(3, 2)
    assert D.world() == (0, 1)
    assert D.gather_rows(x) is x
    assert D.gather_parts(x).shape == (1, 3, 2)
    i, v, (row,) = D.best_row(torch.tensor([3.0, float("nan"), 1.0]), [x])
    assert (i, v) == (2, 1.0) and torch.equal(row, x[2])


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import hmc_oracle as ho
    from paper_2202_07663_gb300 import distributed as D
    from paper_2202_07663_gb300.hmc import DualAveraging
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        # rows of a global array, uneven shards
        n, d = 11, 3
        full = torch.arange(n * d, dtype=torch.float64).reshape(n, d)
        lo, hi = D.shard(n, rank, world)
        res["rows"] = D.gather_rows(full[lo:hi]).numpy()
        res["rows_known"] = D.gather_rows(full[lo:hi], row_counts=D.counts(n, world)).numpy()
        # best start: rank 0 holds NaN and 5, rank 1 holds 2 twice (tie -> first),
        # rank 2 (if any) holds 2 as well (tie -> lower rank wins)
        obj = {0: [float("nan"), 5.0], 1: [7.0, 2.0, 2.0], 2: [2.0]}[rank]
        th = torch.tensor([[10.0 * rank + i, -1.0] for i in range(len(obj))], dtype=torch.float32)
        z = torch.tensor([[100.0 * rank + i] for i in range(len(obj))], dtype=torch.float64)
        i, v, (tr, zr) = D.best_row(torch.tensor(obj, dtype=torch.float64), [th, z])
        res["best"] = (i, v, tr.numpy(), tr.dtype, zr.numpy())
        # nothing finite anywhere
        i, v, (tr,) = D.best_row(torch.tensor([float("inf")], dtype=torch.float64), [th[:1]])
        res["none"] = (i, v, bool(torch.isnan(tr).all()))
        # dual averaging on the mean acceptance over all chains
        B = 50
        rng = np.random.default_rng(5)
        accept = torch.from_numpy(rng.uniform(0, 1, size=(40, B)))
        lo, hi = D.shard(B, rank, world)
        da = DualAveraging(0.3)
        res["eps"] = [da.update(float(D.mean(accept[k, lo:hi], row_counts=D.counts(B, world)))) for k in range(40)]
        # ChEES gradient from gathered rows of every chain
        dd = 4
        q_prev = torch.from_numpy(rng.normal(size=(B, dd)))
        q_prop = torch.from_numpy(rng.normal(size=(B, dd)))
        p_prop = torch.from_numpy(rng.normal(size=(B, dd)))
        w = torch.from_numpy(rng.uniform(0, 1, size=B))
        g = [D.gather_rows(x[lo:hi], row_counts=D.counts(B, world)).numpy() for x in (q_prev, q_prop, p_prop, w)]
        res["chees"] = ho.chees_grad_log_t(g[0], g[1], g[2] * 1.0, g[3], 0.7)
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_agree_with_one_process(world):
    from oracle import hmc_oracle as ho
    from paper_2202_07663_gb300.hmc import DualAveraging
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    n, d = 11, 3
    full = np.arange(n * d, dtype=np.float64).reshape(n, d)
    for r in range(world):
        np.testing.assert_array_equal(res[r]["rows"], full)
        np.testing.assert_array_equal(res[r]["rows_known"], full)
        i, v, tr, dt, zr = res[r]["best"]
        # global order: rank 0 [nan, 5], rank 1 [7, 2, 2], ... -> global index 3 (rank 1, local 1)
        assert (i, v) == (3, 2.0) and dt == torch.float32
        np.testing.assert_array_equal(tr, [11.0, -1.0])
        np.testing.assert_array_equal(zr, [101.0])
        assert res[r]["none"] == (-1, float("inf"), True)
    # every rank holds the same adapted step sizes, equal to one process's
    rng = np.random.default_rng(5)
    accept = rng.uniform(0, 1, size=(40, 50))
    da = DualAveraging(0.3)
    eps1 = [da.update(float(torch.from_numpy(accept[k]).mean())) for k in range(40)]
    for r in range(world):
        assert res[r]["eps"] == res[0]["eps"]
    np.testing.assert_allclose(res[0]["eps"], eps1, rtol=1e-12)
    q_prev, q_prop, p_prop = (rng.normal(size=(50, 4)) for _ in range(3))
    w = rng.uniform(0, 1, size=50)
    want = ho.chees_grad_log_t(q_prev, q_prop, p_prop, w, 0.7)
    for r in range(world):
        assert res[r]["chees"] == want
