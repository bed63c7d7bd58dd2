"""Parity of the device explorer pool (pfsp_solve) with the CPU oracle.

* Finding mode (incumbent from NEH): the optimal makespan must equal the
  oracle's (and brute force where n <= 10); the returned permutation must be
  valid and reach it.
* Proof mode (incumbent fixed at the optimum, or below it as in the paper's
  fixed-tree experiments): the search tree is fixed, so the decomposed-node and
  bounded-children counts must equal the sequential oracle's exactly, whatever
  the number of explorers and the work stealing that happened.
"""
import json
import os

import numpy as np
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


def _check_perm(p, r):
    n = p.shape[0]
    assert sorted(r["perm"].tolist()) == list(range(n))
    assert orc.makespan(p, r["perm"]) == r["cmax"]


@pytest.mark.parametrize("seed", range(1, 11))
def test_n10_m5_lb1_neh_equals_brute_force(pf, seed):
    p = inputs.make_instance(10, 5, seed)
    inst = pf.pfsp_load_instance(p)
    r = pf.pfsp_solve(inst, bound=pf.PFSP_LB1)
    opt, _ = orc.brute_force(p)
    assert r["outcome"] == pf.PFSP_OPTIMAL
    assert r["cmax"] == opt
    _check_perm(p, r)


@pytest.mark.parametrize("n,m,bound,seed", [
    (12, 5, 1, 1), (12, 5, 1, 2), (13, 4, 1, 3), (11, 10, 2, 4), (10, 20, 2, 5), (12, 8, 2, 6),
    (9, 3, 2, 7), (14, 5, 1, 8),
])
def test_proof_mode_counts_equal_oracle(pf, n, m, bound, seed):
    p = inputs.make_instance(n, m, seed)
    want = orc.bb_solve(p, bound=bound)
    opt = want["cmax"]
    proof = orc.bb_solve(p, bound=bound, init_ub=opt)
    inst = pf.pfsp_load_instance(p)
    r = pf.pfsp_solve(inst, bound=bound, init_ub=opt)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert r["cmax"] == opt
    assert (r["decomposed"], r["bounded_children"]) == (proof["decomposed"], proof["bounded"])
    assert r["leaves"] == proof["leaves"] and r["pruned"] == proof["pruned"]
    g = pf.pfsp_solve(inst, bound=bound)
    assert g["outcome"] == pf.PFSP_OPTIMAL and g["cmax"] == opt
    _check_perm(p, g)


@pytest.mark.parametrize("bound", [1, 2])
def test_capped_minmin_proof_counts(pf, bound):
    p = inputs.make_instance(12, 6, 31 + bound)
    opt = orc.bb_solve(p, bound=bound)["cmax"]
    proof = orc.bb_solve(p, bound=bound, init_ub=opt, capped=True)
    inst = pf.pfsp_load_instance(p)
    r = pf.pfsp_solve(inst, bound=bound, init_ub=opt, branching=pf.PFSP_MINMIN_CAPPED)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (r["decomposed"], r["bounded_children"]) == (proof["decomposed"], proof["bounded"])


@pytest.mark.parametrize("rule", ["MINBRANCH", "MINSUM"])
@pytest.mark.parametrize("n,m,bound,seed", [(15, 5, 1, 46), (13, 8, 2, 45), (14, 6, 2, 48), (13, 8, 2, 49)])
def test_other_branching_rules_proof_counts(pf, rule, n, m, bound, seed):
    # MinBranch / MinSum (Table 4's rules): the proof tree and every counter
    # equal the oracle's; finding mode reaches the oracle's optimum
    br = getattr(pf, "PFSP_" + rule)
    p = inputs.make_instance(n, m, seed)
    opt = orc.bb_solve(p, bound=bound)["cmax"]
    proof = orc.bb_solve(p, bound=bound, init_ub=opt, branching=getattr(orc, rule))
    inst = pf.pfsp_load_instance(p)
    r = pf.pfsp_solve(inst, bound=bound, init_ub=opt, branching=br)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (r["decomposed"], r["bounded_children"]) == (proof["decomposed"], proof["bounded"])
    assert r["leaves"] == proof["leaves"] and r["pruned"] == proof["pruned"]
    g = pf.pfsp_solve(inst, bound=bound, branching=br)
    assert g["outcome"] == pf.PFSP_OPTIMAL and g["cmax"] == opt
    _check_perm(p, g)


@pytest.mark.parametrize("n,m,bound,seed", [(12, 6, 1, 20), (13, 6, 1, 22), (14, 8, 1, 21), (12, 10, 1, 22),
                                             (12, 8, 2, 42), (36, 3, 1, 4)])
def test_heads_tails_refinement_proof_counts(pf, n, m, bound, seed):
    # lb1_minht: the refined LB1 (and LB2 over it); proof trees and counters
    # equal the oracle's with the same refinement, finding mode its optimum
    p = inputs.make_instance(n, m, seed)
    if n > 20:
        ub = orc.lb1(p, [], [], minht=True) + 4  # a tight incumbent keeps the oracle's tree small
        want = orc.bb_solve(p, bound=bound, init_ub=ub, minht=True, node_limit=3_000_000)
        assert want["outcome"] != orc.LIMIT_NODES
        r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=bound, init_ub=ub, lb1_minht=1)
        assert r["outcome"] == want["outcome"] and r["cmax"] == want["cmax"]
        if want["outcome"] == orc.PROVEN_NO_BETTER:
            assert (r["decomposed"], r["bounded_children"]) == (want["decomposed"], want["bounded"])
        return
    opt = orc.bb_solve(p, bound=bound)["cmax"]
    proof = orc.bb_solve(p, bound=bound, init_ub=opt, minht=True)
    inst = pf.pfsp_load_instance(p)
    r = pf.pfsp_solve(inst, bound=bound, init_ub=opt, lb1_minht=1)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (r["decomposed"], r["bounded_children"]) == (proof["decomposed"], proof["bounded"])
    assert r["leaves"] == proof["leaves"] and r["pruned"] == proof["pruned"]
    g = pf.pfsp_solve(inst, bound=bound, lb1_minht=1)
    assert g["outcome"] == pf.PFSP_OPTIMAL and g["cmax"] == opt
    _check_perm(p, g)


def test_fixed_tree_below_optimum(pf):
    # the paper's fixed-tree runs start from an incumbent at or below the optimum
    p = inputs.make_instance(13, 6, 9)
    opt = orc.bb_solve(p, bound=1)["cmax"]
    for ub in (opt - 20, opt - 3, opt, opt + 1):
        want = orc.bb_solve(p, bound=1, init_ub=ub)
        r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=1, init_ub=ub)
        assert r["outcome"] == want["outcome"]
        assert r["cmax"] == want["cmax"]
        if want["outcome"] == orc.PROVEN_NO_BETTER:
            assert (r["decomposed"], r["bounded_children"]) == (want["decomposed"], want["bounded"])


@pytest.mark.parametrize("warps", [1, 2, 5, 0])
def test_counts_independent_of_pool_size(pf, warps):
    p = inputs.make_instance(12, 10, 17)
    opt = orc.bb_solve(p, bound=2)["cmax"]
    proof = orc.bb_solve(p, bound=2, init_ub=opt)
    r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=2, init_ub=opt, warps_per_sm=warps)
    assert (r["decomposed"], r["bounded_children"]) == (proof["decomposed"], proof["bounded"])


def test_more_than_32_jobs(pf):
    # two-word job masks; a tight incumbent keeps the tree small for the oracle
    n, m = 36, 3
    p = inputs.make_instance(n, m, 4)
    root = orc.lb1(p, [], [])
    for bound in (1, 2):
        ub = root + 4
        want = orc.bb_solve(p, bound=bound, init_ub=ub, node_limit=3_000_000)
        assert want["outcome"] != orc.LIMIT_NODES
        r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=bound, init_ub=ub)
        assert r["outcome"] == want["outcome"] and r["cmax"] == want["cmax"]
        if want["outcome"] == orc.PROVEN_NO_BETTER:
            assert (r["decomposed"], r["bounded_children"]) == (want["decomposed"], want["bounded"])
        else:
            _check_perm(p, r)


def test_degenerate_instances(pf):
    for n, m in [(1, 1), (1, 5), (2, 1), (2, 2), (3, 1), (5, 1)]:
        p = inputs.make_instance(n, m, 3)
        r = pf.pfsp_solve(pf.pfsp_load_instance(p), bound=2)
        assert r["cmax"] == orc.brute_force(p)[0]
        assert r["outcome"] == pf.PFSP_OPTIMAL
        _check_perm(p, r)


def test_limits(pf):
    # a 50 x 20 instance from its NEH schedule takes far longer than the limits
    p = inputs.make_instance(50, 20, 1)
    neh, _ = orc.neh(p)
    inst = pf.pfsp_load_instance(p)
    r = pf.pfsp_solve(inst, bound=1, node_limit=20000)
    assert r["outcome"] == pf.PFSP_LIMIT_NODES
    assert r["decomposed"] >= 20000
    assert r["cmax"] <= neh
    _check_perm(p, r)
    r = pf.pfsp_solve(inst, bound=1, time_limit_s=0.2)
    assert r["outcome"] == pf.PFSP_LIMIT_TIME
    assert r["cmax"] <= neh
    _check_perm(p, r)


@pytest.mark.parametrize("n,m,seed", [(12, 10, 2), (11, 20, 3), (12, 6, 4)])
def test_adjacent_pair_lb2_solve_matches_oracle(pf, n, m, seed):
    # the paper's LB2 may use as few as the m - 1 adjacent machine pairs: the
    # solve is exact (optimum) and its proof-mode tree is the oracle's tree for
    # that bound, node for node
    p = inputs.make_instance(n, m, seed)
    adjacent = [k * (2 * m - k - 1) // 2 for k in range(m - 1)]
    opt = orc.bb_solve(p, bound=orc.LB2)["cmax"]
    want = orc.bb_solve(p, bound=orc.LB2, init_ub=opt, pairs=adjacent)
    inst = pf.pfsp_load_instance(p)
    pf.pfsp_set_lb2_pairs(inst, adjacent)
    r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (r["decomposed"], r["bounded_children"], r["pruned"]) == (want["decomposed"], want["bounded"],
                                                                      want["pruned"])
    assert r["lb2_slots"] <= r["decomposed"]  # one slot per decomposition at most
    f = pf.pfsp_solve(inst, bound=pf.PFSP_LB2)
    assert f["cmax"] == opt
    _check_perm(p, f)


def test_phase_timers_and_slot_counter(pf):
    # the opt-in phase timers fill the cycle counters without changing the
    # search; without them the counters stay zero.  The LB2 slot counter is
    # one per decomposition with unscheduled jobs (ceil(45 / 32) = 2 at m = 10).
    g = [r for r in json.load(open(GOLDEN))["results"] if r["seed"] == 1][0]
    inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, 1))
    off = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"])
    on = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"], phase_timers=1)
    assert off["decomposed"] == on["decomposed"] == g["proof_decomposed"]
    assert sum(off["phase_cycles"].values()) == 0
    ph = on["phase_cycles"]
    assert ph["lb1"] > 0 and ph["lb2"] > 0 and ph["select"] > 0 and ph["branch"] > 0
    assert off["lb2_slots"] == on["lb2_slots"] == 2 * g["proof_decomposed"]


def test_invalid_options(pf):
    p = inputs.make_instance(8, 4, 1)
    inst = pf.pfsp_load_instance(p)
    for bad in (dict(bound=3), dict(branching=5), dict(branching=-1), dict(node_limit=-1),
                dict(branching=pf.PFSP_MINSUM, learned=pf.PFSP_EARLY_EXIT), dict(lb1_minht=2)):
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_solve(inst, **bad)
        assert e.value.code == pf.PFSP_ERR_INVALID


def _golden():
    if not os.path.exists(GOLDEN):
        pytest.skip("oracle results not generated (tests/golden/make_solve_golden.py)")
    with open(GOLDEN) as f:
        return json.load(f)["results"]


@pytest.mark.parametrize("seed", range(1, 11))
def test_n20_m10_lb2_optimum_and_proof_counts(pf, seed):
    g = {r["seed"]: r for r in _golden()}[seed]
    p = inputs.make_instance(20, 10, seed)
    inst = pf.pfsp_load_instance(p)
    r = pf.pfsp_solve(inst, bound=2, init_ub=g["optimum"])
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (r["decomposed"], r["bounded_children"]) == (g["proof_decomposed"], g["proof_bounded"])
    rc = pf.pfsp_solve(inst, bound=2, init_ub=g["optimum"], branching=pf.PFSP_MINMIN_CAPPED)
    assert rc["decomposed"] == g["proof_capped_decomposed"]
    f = pf.pfsp_solve(inst, bound=2)
    assert f["outcome"] == pf.PFSP_OPTIMAL and f["cmax"] == g["optimum"]
    _check_perm(p, f)


@pytest.mark.parametrize("min_steal", [2.0, 40320.0, 1e30])
def test_minimum_split_keeps_the_proof_tree(pf, min_steal):
    # a victim splits its interval only when it holds at least min_steal
    # leaves (the work stealing of Section 3.4 with a minimum split); the
    # proof's tree is the same whatever the threshold, and above every
    # interval's length (20! < 1e30) no steal is granted at all
    g = {r["seed"]: r for r in _golden()}[10]
    inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, 10))
    r = pf.pfsp_solve(inst, bound=2, init_ub=g["optimum"], min_steal=min_steal)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (r["decomposed"], r["bounded_children"]) == (g["proof_decomposed"], g["proof_bounded"])
    if min_steal > 1e20:
        assert r["steals"] == 0
    else:
        assert r["steals"] > 0


def test_steal_wait_expiry_returns_timeout(pf):
    # a thief's bounded wait for a victim's answer (the steal handshake of
    # Section 3.4) made to run out on purpose: with one poll allowed, the first
    # request that the victim does not answer at once ends the solve with
    # PFSP_ERR_TIMEOUT and nothing written; nothing faults or hangs, and the
    # next solve, with the default limit, runs normally on the same context
    path = os.path.join(os.path.dirname(__file__), "golden", "solve_20x10_lb2.json")
    g = {r["seed"]: r for r in json.load(open(path))["results"]}[7]
    inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, 7))
    try:
        pf.pfsp_set_steal_wait_limit(1)
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"])
        assert e.value.code == pf.PFSP_ERR_TIMEOUT
    finally:
        pf.pfsp_set_steal_wait_limit(0)
    r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"])
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER and r["decomposed"] == g["proof_decomposed"]
    with pytest.raises(pf.PfspError):
        pf.pfsp_set_steal_wait_limit(-1)
