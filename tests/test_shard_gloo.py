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


def test_single_process_rate_is_local():
    from paper_2012_09511_gb300 import shard
    rate, slowest, total = shard.whole_job_rate(0.5, 1000)
    assert (rate, slowest, total) == (2000.0, 0.5, 1000.0)
