"""Heuristic threads beside the explorer pool (Section 4.2), on the GPU.

The host threads' schedules lower the explorers' incumbent through
host-mapped memory, and the explorers' nodes are promoted to their starting
points.  Whatever they find, the solve stays exact: finding mode ends at the
oracle's optimum with a schedule of that makespan; proof mode (incumbent at
the optimum, which nothing can beat) explores exactly the oracle's tree.
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
from paper_2012_09511_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "solve_20x10_lb2.json")


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import pfsp
    return pfsp


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return {r["seed"]: r for r in json.load(f)["results"]}


def _check(p, r, c):
    assert r["cmax"] == c
    assert sorted(r["perm"].tolist()) == list(range(p.shape[0]))
    assert orc.makespan(p, r["perm"]) == c


@pytest.mark.parametrize("seed", [1, 3, 5, 7, 8, 10])
@pytest.mark.parametrize("threads", [1, 4])
def test_finding_mode_reaches_the_optimum(pf, gold, seed, threads):
    g = gold[seed]
    p = inputs.make_instance(20, 10, seed)
    inst = pf.pfsp_load_instance(p)
    for rule in (pf.PFSP_MINMIN, pf.PFSP_MINBRANCH):
        r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, branching=rule, heuristic_threads=threads,
                          heuristic_seed=seed)
        assert r["outcome"] == pf.PFSP_OPTIMAL
        _check(p, r, g["optimum"])
        assert r["heuristic_cmax"] >= g["optimum"]


def test_proof_mode_tree_is_unchanged(pf, gold):
    for seed in (1, 3, 7):
        g = gold[seed]
        inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, seed))
        r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"], heuristic_threads=2)
        assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER and r["cmax"] == g["optimum"]
        assert (r["decomposed"], r["bounded_children"]) == (g["proof_decomposed"], g["proof_bounded"])
        assert r["heuristic_improvements"] == 0 and r["heuristic_cmax"] == pf.INT32_MAX


@pytest.mark.parametrize("kind", [1, 2])
def test_beam_search_threads_reach_the_optimum(pf, gold, kind):
    # heuristic_kind 1: beam search below the promoted explorer nodes; 2: both searches
    for seed in (1, 4, 7):
        g = gold[seed]
        p = inputs.make_instance(20, 10, seed)
        r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=pf.PFSP_LB2, heuristic_threads=4, heuristic_kind=kind,
                          heuristic_seed=seed)
        assert r["outcome"] == pf.PFSP_OPTIMAL
        _check(p, r, g["optimum"])
        assert r["heuristic_cmax"] >= g["optimum"]
        if seed == 4:
            # the beam threads start from the promoted nodes (whether they beat
            # the explorers' own incumbent depends on the run)
            assert r["promoted"] > 0 and r["snapshots"] > 0


def test_long_solve_promotes_explorer_nodes(pf, gold):
    # seed 4 takes tens of milliseconds from NEH: several snapshot rounds
    g = gold[4]
    p = inputs.make_instance(20, 10, 4)
    r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=pf.PFSP_LB2, heuristic_threads=4, heuristic_seed=1)
    assert r["outcome"] == pf.PFSP_OPTIMAL
    _check(p, r, g["optimum"])
    info = {k: r[k] for k in ("kernel_seconds", "snapshots", "promoted", "heuristic_improvements",
                              "heuristic_cmax")}
    assert r["snapshots"] > 0 and r["promoted"] > 0, info
    assert r["heuristic_improvements"] > 0 and r["heuristic_cmax"] < orc.neh(p)[0], info


def test_limit_stop_returns_the_best_schedule(pf, gold):
    p = inputs.make_instance(20, 10, 4)
    neh_c = orc.neh(p)[0]
    r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=pf.PFSP_LB2, node_limit=5000, heuristic_threads=2)
    assert r["outcome"] == pf.PFSP_LIMIT_NODES
    assert gold[4]["optimum"] <= r["cmax"] <= neh_c
    _check(p, r, r["cmax"])


def test_checkpoint_after_heuristic_segment_resumes_exactly(pf, gold):
    g = gold[7]
    p = inputs.make_instance(20, 10, 7)
    inst = pf.pfsp_load_instance(p)
    a = pf.pfsp_solve_resumable(inst, bound=pf.PFSP_LB2, node_limit=20000, heuristic_threads=2)
    assert a["outcome"] == pf.PFSP_LIMIT_NODES and a["checkpoint"]
    _check(p, a, a["cmax"])
    b = pf.pfsp_solve_resumable(inst, bound=pf.PFSP_LB2, resume=a["checkpoint"])
    assert b["outcome"] == pf.PFSP_OPTIMAL
    _check(p, b, g["optimum"])


def test_heuristic_options_validation(pf):
    p = inputs.make_instance(8, 4, 1)
    inst = pf.pfsp_load_instance(p)
    for bad in (dict(heuristic_threads=-1), dict(heuristic_threads=1, heuristic_kind=3)):
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_solve(inst, **bad)
        assert e.value.code == pf.PFSP_ERR_INVALID
    with pytest.raises(pf.PfspError) as e:
        pf.pfsp_solve_batch([inst], heuristic_threads=1)
    assert e.value.code == pf.PFSP_ERR_UNSUPPORTED
    with pytest.raises(pf.PfspError) as e:
        pf.pfsp_solve_noalloc(p, heuristic_threads=1)
    assert e.value.code == pf.PFSP_ERR_UNSUPPORTED
    # the heads and tails refinement runs in its own kernel, beside neither
    for bad in (dict(lb1_minht=1, heuristic_threads=1),):
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_solve(inst, **bad)
        assert e.value.code == pf.PFSP_ERR_UNSUPPORTED
    with pytest.raises(pf.PfspError) as e:
        pf.pfsp_solve_batch([inst], lb1_minht=1)
    assert e.value.code == pf.PFSP_ERR_UNSUPPORTED
    with pytest.raises(pf.PfspError) as e:
        pf.pfsp_solve_noalloc(p, lb1_minht=1)
    assert e.value.code == pf.PFSP_ERR_UNSUPPORTED
