"""The multi-rank path of the bounding benchmark on CPU: two gloo ranks.

Each rank draws its own node batch (different seeds, so the shards differ)
and reports a time and a unit count; the whole-job rate must be the summed
units over the slowest rank's time, identical on both ranks.
"""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_2012_09511_gb300 import inputs, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 20
        perm, d1, d2 = inputs.random_nodes(n, 64, seed=shard.rank_seed(2020, rank), dmax=10)
        units = int(2 * (n - d1.astype(np.int64) - d2.astype(np.int64)).sum())
        seconds = 0.010 * (rank + 1)  # rank 1 is the slow one
        rate, slowest, total = shard.whole_job_rate(seconds, units, device="cpu")
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"units": units, "rate": rate, "slowest": slowest, "total": total,
                       "first_row": perm[0].tolist()}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_weak_scaling(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / ("rank%d.json" % i))) for i in range(world)]
    assert r[0]["first_row"] != r[1]["first_row"]  # each rank bounds its own batch
    total = r[0]["units"] + r[1]["units"]
    for x in r:
        assert x["total"] == total
        assert x["slowest"] == pytest.approx(0.020)
        assert x["rate"] == pytest.approx(total / 0.020)


def _range_rank_main(rank, world, port, out_dir):
    # each rank bounds its range of one shared batch with the oracle (LB1 and
    # full-pair LB2 of every child) and the ranks gather the pieces; no data
    # crosses ranks until the final gather
    import torch.distributed as dist
    import oracle
    from paper_2012_09511_gb300 import inputs, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, m, count = 20, 20, 301
        p = inputs.make_instance(n, m, 2020)
        perm, d1, d2 = inputs.random_nodes(n, count, seed=2020)
        lo, hi = shard.node_range(count, rank, world)
        b1, b2 = oracle.children_bounds_batch(p, perm[lo:hi], d1[lo:hi], d2[lo:hi])
        pieces = [None] * world
        dist.all_gather_object(pieces, (lo, hi, b1.tolist(), b2.tolist()))
        if rank == 0:
            with open(os.path.join(out_dir, "gathered.json"), "w") as f:
                json.dump(pieces, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_split_one_batch_by_range(tmp_path, world):
    import oracle
    from paper_2012_09511_gb300 import inputs
    oracle.build()
    mp.start_processes(_range_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    pieces = json.load(open(tmp_path / "gathered.json"))
    n, m, count = 20, 20, 301
    # the ranges tile [0, count) in rank order
    assert pieces[0][0] == 0 and pieces[-1][1] == count
    assert all(pieces[i][1] == pieces[i + 1][0] for i in range(world - 1))
    got1 = np.concatenate([np.array(x[2], dtype=np.int32).reshape(-1, 2, n) for x in pieces])
    got2 = np.concatenate([np.array(x[3], dtype=np.int32).reshape(-1, 2, n) for x in pieces])
    p = inputs.make_instance(n, m, 2020)
    perm, d1, d2 = inputs.random_nodes(n, count, seed=2020)
    w1, w2 = oracle.children_bounds_batch(p, perm, d1, d2)
    assert (got1 == w1.reshape(count, 2, n)).all() and (got2 == w2.reshape(count, 2, n)).all()


def test_node_range_tiles_the_batch():
    from paper_2012_09511_gb300 import shard
    for count in (0, 1, 7, 301, 4194304):
        for world in (1, 2, 3, 8):
            r = [shard.node_range(count, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == count
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.node_range(10, 2, 2)


def test_single_process_rate_is_local():
    from paper_2012_09511_gb300 import shard
    rate, slowest, total = shard.whole_job_rate(0.5, 1000)
    assert (rate, slowest, total) == (2000.0, 0.5, 1000.0)
