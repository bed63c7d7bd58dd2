"""Checkpoint and resume of the explorer pool (pfsp_solve_resumable).

The paper's coordinator keeps the unexplored intervals and the best solution
in a checkpoint file and restarts from it (Section 4.1).  Here one GPU's
explorer pool stops at a node or time limit, hands back the rest of every
explorer's interval, and a later call resumes from those bytes.

* Proof mode (incumbent fixed at the optimum): every node is decomposed in
  exactly one segment, so the decomposed, bounded and pruned counts of the
  segments add up to the oracle's counts of the whole tree.
* Finding mode: the segments end with the oracle's optimum and a schedule
  that reaches it.
* A checkpoint of another instance or another branching rule is refused.
"""
import json
import os

import pytest

import oracle as orc
from paper_2012_09511_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "solve_20x10_lb2.json")


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import pfsp
    return pfsp


def _segments(pf, inst, limit, max_segments=200, **kw):
    tot = {"decomposed": 0, "bounded_children": 0, "pruned": 0, "leaves": 0}
    ck, segs, r = None, 0, None
    while True:
        r = pf.pfsp_solve_resumable(inst, resume=ck, node_limit=limit, **kw)
        for k in tot:
            tot[k] += r[k]
        segs += 1
        ck = r["checkpoint"]
        if ck is None:
            return r, tot, segs
        assert r["outcome"] == pf.PFSP_LIMIT_NODES
        assert segs < max_segments


@pytest.mark.parametrize("seed,limit", [(1, 5000), (7, 150000), (8, 20000)])
def test_proof_counts_add_up_across_segments(pf, seed, limit):
    g = [r for r in json.load(open(GOLDEN))["results"] if r["seed"] == seed][0]
    inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, seed))
    r, tot, segs = _segments(pf, inst, limit, bound=pf.PFSP_LB2, init_ub=g["optimum"])
    assert segs >= 3
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (tot["decomposed"], tot["bounded_children"], tot["pruned"]) == (
        g["proof_decomposed"], g["proof_bounded"], g["proof_pruned"])


@pytest.mark.parametrize("n,m,bound,seed,capped", [(12, 8, 2, 6, False), (13, 5, 1, 3, True), (12, 10, 2, 17, True)])
def test_proof_counts_small_instances(pf, n, m, bound, seed, capped):
    p = inputs.make_instance(n, m, seed)
    opt = orc.bb_solve(p, bound=bound)["cmax"]
    want = orc.bb_solve(p, bound=bound, init_ub=opt, capped=capped)
    inst = pf.pfsp_load_instance(p)
    br = pf.PFSP_MINMIN_CAPPED if capped else pf.PFSP_MINMIN
    r, tot, segs = _segments(pf, inst, max(500, want["decomposed"] // 6), bound=bound, init_ub=opt, branching=br,
                             learned=pf.PFSP_EARLY_EXIT)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (tot["decomposed"], tot["bounded_children"], tot["pruned"]) == (
        want["decomposed"], want["bounded"], want["pruned"])


def test_finding_mode_reaches_the_optimum(pf):
    g = [r for r in json.load(open(GOLDEN))["results"] if r["seed"] == 7][0]
    p = inputs.make_instance(20, 10, 7)
    inst = pf.pfsp_load_instance(p)
    r, tot, segs = _segments(pf, inst, 100000, bound=pf.PFSP_LB2)
    assert segs >= 2
    assert r["outcome"] == pf.PFSP_OPTIMAL and r["cmax"] == g["optimum"]
    assert sorted(r["perm"].tolist()) == list(range(20)) and orc.makespan(p, r["perm"]) == g["optimum"]


def test_checkpoint_is_bytes_and_is_checked(pf, tmp_path):
    g = [r for r in json.load(open(GOLDEN))["results"] if r["seed"] == 4][0]
    inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, 4))
    r = pf.pfsp_solve_resumable(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"], node_limit=50000)
    ck = r["checkpoint"]
    assert r["outcome"] == pf.PFSP_LIMIT_NODES and ck[:8] == b"PFSPCKP1"
    path = tmp_path / "pool.ckpt"
    path.write_bytes(ck)
    r2 = pf.pfsp_solve_resumable(inst, resume=path.read_bytes(), bound=pf.PFSP_LB2, node_limit=50000)
    assert r2["outcome"] in (pf.PFSP_LIMIT_NODES, pf.PFSP_PROVEN_NO_BETTER)
    other = pf.pfsp_load_instance(inputs.make_instance(20, 5, 4))
    with pytest.raises(pf.PfspError):
        pf.pfsp_solve_resumable(other, resume=ck, bound=pf.PFSP_LB2)
    with pytest.raises(pf.PfspError):  # another branching rule
        pf.pfsp_solve_resumable(inst, resume=ck, bound=pf.PFSP_LB2, branching=pf.PFSP_MINMIN_CAPPED)
    with pytest.raises(pf.PfspError):  # truncated
        pf.pfsp_solve_resumable(inst, resume=ck[:-5], bound=pf.PFSP_LB2)


@pytest.mark.parametrize("workers,seed,limit", [(3, 1, 4000), (2, 8, 20000), (4, 5, 3000)])
def test_pools_under_the_coordinator_decompose_every_node_once(pf, workers, seed, limit):
    # several explorer pools (taking turns on this GPU) share the tree through
    # the work-unit coordinator of Algorithm 1: in proof mode the counters of
    # all their segments add up to the oracle's counts of the whole tree
    from paper_2012_09511_gb300 import coordinator as co
    g = [r for r in json.load(open(GOLDEN))["results"] if r["seed"] == seed][0]
    inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, seed))
    ws = [co.PoolWorker(pf, inst, bound=pf.PFSP_LB2, cap=g["optimum"], node_limit=limit) for _ in range(workers)]
    coord = co.Coordinator(20, ub=g["optimum"])
    co.solve_with_workers(ws, coord)
    tot = {k: sum(w.counts[k] for w in ws) for k in ws[0].counts}
    assert (tot["decomposed"], tot["bounded_children"], tot["pruned"]) == (
        g["proof_decomposed"], g["proof_bounded"], g["proof_pruned"])
    assert coord.steals > 0 and coord.ub == g["optimum"] and coord.best_perm is None
    assert all(w.segments > 1 for w in ws)


def test_pools_under_the_coordinator_find_the_optimum(pf):
    from paper_2012_09511_gb300 import coordinator as co
    g = [r for r in json.load(open(GOLDEN))["results"] if r["seed"] == 7][0]
    p = inputs.make_instance(20, 10, 7)
    inst = pf.pfsp_load_instance(p)
    ub0 = g["optimum"] + 40
    ws = [co.PoolWorker(pf, inst, bound=pf.PFSP_LB2, cap=ub0, node_limit=60000) for _ in range(3)]
    coord = co.Coordinator(20, ub=ub0)
    co.solve_with_workers(ws, coord)
    assert coord.ub == g["optimum"]
    assert sorted(coord.best_perm) == list(range(20)) and orc.makespan(p, coord.best_perm) == g["optimum"]
