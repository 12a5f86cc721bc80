"""Host logic of the continuous-batching scheduler (no GPU): admission by the
device-memory budget in arrival order, round-robin batches within the scratch
arena and segment limits, every vector scheduled exactly once, budget
returned on completion."""
import numpy as np
import pytest

from paper_2202_07663_gb300.serving import IO_BYTES_PER_VECTOR, Job, Scheduler


def seg_bytes(job, n):
    return 1000 * n + 4096          # stand-in for the batcher's per-segment scratch


def test_admission_respects_budget_and_order():
    s = Scheduler(budget_bytes=3 * (1000 + 100 * IO_BYTES_PER_VECTOR), arena_bytes=10 ** 9, max_segments=8,
                  chunk=64, segment_bytes=seg_bytes)
    jobs = [Job(i, 0.1 * i, 100, 1000) for i in range(5)]
    for j in jobs:
        s.arrive(j)
    got = s.admit(0.0)
    assert [j.index for j in got] == [0, 1, 2]
    assert s.used <= s.budget
    assert [j.index for j in s.waiting] == [3, 4]
    with pytest.raises(ValueError):
        s.arrive(Job(9, 0.0, 10 ** 9, 0))


def test_round_robin_chunks_cover_every_vector_once():
    rng = np.random.default_rng(0)
    s = Scheduler(budget_bytes=10 ** 12, arena_bytes=300_000, max_segments=4, chunk=64, segment_bytes=seg_bytes)
    jobs = [Job(i, 0.0, int(rng.integers(1, 300)), 5000) for i in range(9)]
    for j in jobs:
        s.arrive(j)
    s.admit(0.0)
    seen = {j.index: np.zeros(j.B, int) for j in jobs}
    first_batch = None
    batches = 0
    while True:
        segs = s.next_batch()
        if not segs:
            break
        batches += 1
        if first_batch is None:
            first_batch = [j.index for j, _, _ in segs]
        assert len(segs) <= 4
        assert sum(seg_bytes(j, c) for j, _, c in segs) <= 300_000
        assert len({j.index for j, _, _ in segs}) == len(segs)      # at most one range per job
        for j, a, c in segs:
            seen[j.index][a:a + c] += 1
        for j in list(s.active):
            if j.remaining == 0:
                s.complete(j, float(batches))
    assert all((v == 1).all() for v in seen.values())
    assert first_batch == [0, 1, 2, 3]
    assert s.idle() and s.used == 0 and len(s.finished) == 9


def test_completion_frees_budget_for_waiting_requests():
    s = Scheduler(budget_bytes=2000 + 10 * IO_BYTES_PER_VECTOR, arena_bytes=10 ** 9, max_segments=8, chunk=64,
                  segment_bytes=seg_bytes)
    a, b = Job(0, 0.0, 10, 2000), Job(1, 0.0, 10, 2000)
    s.arrive(a)
    s.arrive(b)
    assert [j.index for j in s.admit(0.0)] == [0]
    s.next_batch()
    s.complete(a, 1.0)
    assert [j.index for j in s.admit(1.0)] == [1]


def test_arena_limit_halves_a_chunk():
    s = Scheduler(budget_bytes=10 ** 12, arena_bytes=40_000, max_segments=8, chunk=64, segment_bytes=seg_bytes)
    s.arrive(Job(0, 0.0, 64, 0))
    s.admit(0.0)
    segs = s.next_batch()
    assert segs[0][2] == 32 and seg_bytes(None, 32) <= 40_000


def test_admission_limited_to_what_the_next_batches_need():
    """With max_ready, no more than that many admitted jobs wait with vectors
    still to schedule; a job whose vectors are all scheduled frees its slot
    (its budget stays held until it completes)."""
    s = Scheduler(budget_bytes=10 ** 12, arena_bytes=10 ** 9, max_segments=2, chunk=1000, segment_bytes=seg_bytes)
    for i in range(6):
        s.arrive(Job(i, 0.0, 50, 1000))
    assert [j.index for j in s.admit(0.0, max_ready=3)] == [0, 1, 2]
    assert [j.index for j in s.admit(0.0, max_ready=3)] == []
    segs = s.next_batch()                   # jobs 0 and 1, all their vectors
    assert [j.index for j, _, _ in segs] == [0, 1] and all(c == 50 for _, _, c in segs)
    assert [j.index for j in s.admit(0.0, max_ready=3)] == [3, 4]
    assert [j.index for j in s.waiting] == [5]
    used = s.used
    s.complete(segs[0][0], 1.0)
    assert s.used == used - segs[0][0].bytes
