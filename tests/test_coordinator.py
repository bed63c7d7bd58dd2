"""The work-unit coordinator of Section 4.1 (Algorithm 1) on the CPU.

* Factoradic conversion and the checkpoint bytes round-trip.
* Work-unit intersection (Eq. 3 and 4) equals the set intersection, checked
  by brute force on small leaf ranges.
* With stand-in workers that consume leaves from the left of their units,
  the coordinator hands every leaf of [0, n!) to exactly one worker, divides
  the largest unit when a worker runs dry, and spreads the best incumbent;
  once in one process and once over two and three gloo ranks.
"""
import json
import os
import socket
from math import factorial

import numpy as np
import pytest

from paper_2012_09511_gb300 import coordinator as co


def test_factoradic_round_trip():
    for n in (1, 4, 6):
        for x in range(factorial(n)):
            d = co.to_factoradic(n, x)
            assert all(0 <= d[i] < n - i for i in range(n))
            assert co.from_factoradic(d) == x
    big = factorial(30) - 12345
    assert co.from_factoradic(co.to_factoradic(30, big)) == big


def test_checkpoint_bytes_round_trip():
    n = 7
    iv = [(0, 13, -1), (100, 777, 3), (4000, factorial(n), 0)]
    buf = co.pack_checkpoint(n, 5, 2, 1, 400, 390, iv, best_perm=list(range(n)))
    assert buf[:8] == b"PFSPCKP1" and len(buf) == 104 + 3 * co.RECORD_BYTES
    head, back = co.unpack_checkpoint(buf)
    assert back == iv
    assert (head["n"], head["m"], head["bound"], head["branching"], head["cap"], head["ub"]) == (n, 5, 2, 1, 400, 390)
    assert head["best_perm"] == list(range(n))
    with pytest.raises(ValueError):
        co.pack_checkpoint(n, 5, 2, 0, 1, 1, [(5, 5, -1)])


def _leaves(unit):
    s = set()
    for iv in unit:
        s.update(range(iv[0], iv[1]))
    return s


def _random_unit(rng, hi, k):
    cuts = sorted(set(int(x) for x in rng.integers(0, hi + 1, size=2 * k)))
    return [(cuts[i], cuts[i + 1], -1) for i in range(0, len(cuts) - 1, 2) if cuts[i] < cuts[i + 1]]


def test_intersection_is_set_intersection():
    rng = np.random.default_rng(3)
    for _ in range(300):
        w = _random_unit(rng, 120, int(rng.integers(1, 6)))
        c = [(a, b) for a, b, _ in _random_unit(rng, 120, int(rng.integers(1, 6)))]
        got = co.intersect(w, c)
        assert _leaves(got) == _leaves(w) & _leaves(c)
        assert all(got[i][1] <= got[i + 1][0] for i in range(len(got) - 1))


def test_intersection_keeps_levels_of_unchanged_starts():
    w = [(10, 50, 4), (60, 90, 2)]
    c = [(10, 30), (70, 90)]
    assert co.intersect(w, c) == [(10, 30, 4), (70, 90, -1)]


class FakeWorker:
    """Consumes up to `budget` leaves from the left of its unit per segment and
    reports an incumbent that improves once; records what it consumed."""

    def __init__(self, budget, kmax=8, better_at=None):
        self.budget, self.kmax, self.better_at = budget, kmax, better_at
        self.consumed, self.counts, self.segments = [], {"decomposed": 0}, 0

    def run(self, unit, ub, best_perm=None):
        self.segments += 1
        left, budget = [], self.budget
        for a, b, lvl in unit:
            take = min(budget, b - a)
            if take:
                self.consumed.append((a, a + take))
                budget -= take
            if a + take < b:
                left.append((a + take, b, lvl if take == 0 else 7))
        self.counts["decomposed"] += self.budget - budget
        if self.better_at is not None and self.segments == self.better_at:
            return left, min(ub, 1000), [0, 1, 2]
        return left, ub, None


def _check_partition(consumed, total):
    consumed = sorted(consumed)
    assert consumed[0][0] == 0 and consumed[-1][1] == total
    assert all(consumed[i][1] == consumed[i + 1][0] for i in range(len(consumed) - 1))


@pytest.mark.parametrize("workers,budget", [(1, 50), (3, 7), (4, 40), (5, 1)])
def test_every_leaf_goes_to_exactly_one_worker(workers, budget):
    n = 5  # 120 leaves
    ws = [FakeWorker(budget, better_at=1 if i == 1 else None) for i in range(workers)]
    coord = co.Coordinator(n, ub=2000)
    co.solve_with_workers(ws, coord)
    _check_partition([iv for w in ws for iv in w.consumed], factorial(n))
    assert sum(w.counts["decomposed"] for w in ws) == factorial(n)
    if workers > 1:
        assert coord.steals > 0 and all(w.consumed for w in ws)
        assert coord.ub == 1000 and coord.best_perm == [0, 1, 2]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = FakeWorker(budget=5 + 3 * rank, kmax=4, better_at=2 if rank == world - 1 else None)
        coord, counts = co.run_ranks(w, lambda: co.Coordinator(5, ub=2000))
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"consumed": w.consumed, "ub": coord.ub if coord else None,
                       "steals": coord.steals if coord else None}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_coordinator_over_gloo_ranks(tmp_path, world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    outs = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    _check_partition([tuple(iv) for o in outs for iv in o["consumed"]], 120)
    assert all(o["consumed"] for o in outs)
    assert outs[0]["ub"] == 1000 and outs[0]["steals"] > 0
