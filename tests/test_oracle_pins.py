"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints for its worked examples (fixtures under tests/golden/), closed
forms (m = 1, Johnson's rule for m = 2), exhaustive enumeration on tiny
inputs, and invariants (every bound is at most the makespan of every
completion; bounds of complete schedules are exact).  Runs on the CPU only.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_2012_09511_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- Eq. 1 ----

def test_makespan_hand_example():
    # two jobs, two machines: job 0 = (3, 2), job 1 = (1, 4).
    # order (0, 1): machine 1 ends 3 then 4; machine 2 ends 5 then max(5, 4) + 4 = 9.
    # order (1, 0): machine 1 ends 1 then 4; machine 2 ends 5 then max(5, 4) + 2 = 7.
    p = np.array([[3, 2], [1, 4]])
    assert orc.makespan(p, [0, 1]) == 9
    assert orc.makespan(p, [1, 0]) == 7


def test_makespan_single_machine_is_total_work():
    for seed in range(5):
        p = inputs.make_instance(7, 1, seed)
        for perm in (np.arange(7), np.arange(7)[::-1]):
            assert orc.makespan(p, perm) == int(p.sum())


def test_makespan_single_job_is_row_sum():
    p = inputs.make_instance(1, 6, 3)
    assert orc.makespan(p, [0]) == int(p.sum())


def test_makespan_lower_envelopes():
    # C_max >= every machine's total work plus the least head and tail around it
    for seed in range(5):
        p = inputs.make_instance(6, 4, seed).astype(np.int64)
        perm = np.random.default_rng(seed).permutation(6)
        c = orc.makespan(p, perm)
        for k in range(4):
            assert c >= p[:, k].sum()
        assert c >= p.sum(axis=1).max()


# ---------------------------------------------------------------- Johnson --

@pytest.mark.parametrize("seed", range(8))
def test_johnson_is_optimal_for_two_machines(seed):
    p = inputs.make_instance(7, 2, seed)
    cj, order = orc.johnson(p)
    cb, _ = orc.brute_force(p)
    assert cj == cb
    assert orc.makespan(p, order) == cj


@pytest.mark.parametrize("seed", range(6))
def test_johnson_lag_rule_is_optimal(seed):
    # Mitten's extension: for the two-machine problem with time lags, the rule's
    # order attains the minimum over all orders (brute force on 6 jobs).
    rng = np.random.default_rng(100 + seed)
    n = 6
    p = inputs.make_instance(n, 5, seed)
    front = rng.integers(0, 300, 5)
    back = rng.integers(0, 300, 5)
    for k, l in [(0, 1), (0, 4), (1, 3), (2, 4)]:
        g = p[:, k + 1:l].sum(axis=1)
        order = orc.johnson_lag_order(p[:, k], p[:, l], g)
        v_rule = orc.pair_value(p, k, l, front, back, order)
        v_best = min(orc.pair_value(p, k, l, front, back, s) for s in itertools.permutations(range(n)))
        assert v_rule == v_best


# ---------------------------------------------------------------- LB1 ------

def test_fig3_lb1_combination():
    g = golden("fig3_lb1_combination.json")
    assert orc.lb1_combine(g["front"], g["remain"], g["back"]) == g["lb1"]


def test_front_back_remain_hand_example():
    # 3 jobs, 2 machines; sigma1 = (0), sigma2 = (2), job 1 unscheduled.
    p = np.array([[2, 3], [4, 1], [5, 6]])
    assert list(orc.front(p, [0])) == [2, 5]          # job 0 alone: 2, then 2 + 3
    assert list(orc.back(p, [2])) == [11, 6]           # job 2 alone: 5 + 6 from machine 1, 6 from 2
    assert list(orc.remain(p, [1])) == [4, 1]
    # LB1 = max(2 + 4 + 11, 5 + 1 + 6) = 17
    assert orc.lb1(p, [0], [2]) == 17


def test_back_is_reverse_shop_completion():
    # reversibility: the back of sigma2 equals the front of reversed sigma2 on the
    # reversed machine order
    for seed in range(5):
        p = inputs.make_instance(6, 4, seed)
        s2 = [3, 1, 5]
        b = orc.back(p, s2)
        f = orc.front(p[:, ::-1].copy(), s2[::-1])
        assert list(b) == list(f[::-1])


# ---------------------------------------------------------------- bounds ---

def _completions_min(p, s1, s2):
    n = p.shape[0]
    rest = [j for j in range(n) if j not in s1 and j not in s2]
    return min(orc.makespan(p, list(s1) + list(mid) + list(s2)) for mid in itertools.permutations(rest))


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_bounds_valid_exhaustive_small(m):
    # LB1 <= LB2 <= best completion, for every node of a 5-job instance
    p = inputs.make_instance(5, m, 7 + m)
    perm, d1, d2 = inputs.all_nodes_small(5)
    for i in range(len(d1)):
        s1 = list(perm[i, :d1[i]])
        s2 = list(perm[i, 5 - d2[i]:])
        a = orc.lb1(p, s1, s2)
        b = orc.lb2(p, s1, s2)
        best = _completions_min(p, s1, s2)
        assert a <= b <= best, (s1, s2, a, b, best)
        if m == 1:
            assert a == b == best == int(p.sum())


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_minht_valid_and_dominant_exhaustive(m):
    # the refined LB1 never exceeds the best completion of any node of a 5-job
    # instance, never falls below the plain LB1, and differs from it only
    # where sigma1 or sigma2 is empty
    p = inputs.make_instance(5, m, 17 + m)
    perm, d1, d2 = inputs.all_nodes_small(5)
    raised = 0
    for i in range(len(d1)):
        s1 = list(perm[i, :d1[i]])
        s2 = list(perm[i, 5 - d2[i]:])
        a = orc.lb1(p, s1, s2)
        r = orc.lb1(p, s1, s2, minht=True)
        assert a <= r <= _completions_min(p, s1, s2), (s1, s2, a, r)
        if s1 and s2:
            assert r == a
        raised += r > a
    assert m == 1 or raised > 0


def test_minht_hand_example():
    # jobs 0: (1, 2, 3), 1: (4, 1, 1).  At the root the least heads are
    # (0, 1, 3), the least tails (2, 1, 0) and the work (5, 3, 4): the refined
    # LB1 is max(0+5+2, 1+3+1, 3+4+0) = 7, the plain one max(5, 3, 4) = 5.
    # Order (0, 1) has makespan 7 (the bound is tight), order (1, 0) 10.
    p = np.array([[1, 2, 3], [4, 1, 1]], dtype=np.int32)
    assert orc.lb1(p, [], []) == 5
    assert orc.lb1(p, [], [], minht=True) == 7
    assert orc.makespan(p, [0, 1]) == 7 and orc.makespan(p, [1, 0]) == 10
    # job 1 first: the back of sigma2 = () takes job 0's tails (5, 3, 0)
    assert orc.lb1(p, [1], [], minht=True) == max(4 + 1 + 5, 5 + 2 + 3, 6 + 3 + 0)


@pytest.mark.parametrize("m", [2, 4, 7])
def test_minht_single_job_is_exact(m):
    # one unscheduled job and nothing scheduled: the refined LB1 is that
    # job's total work, its makespan
    p = inputs.make_instance(1, m, 3)
    assert orc.lb1(p, [], [], minht=True) == int(p.sum()) == orc.makespan(p, [0])


def test_minht_children_bounds_match_single_nodes():
    n, m = 9, 5
    p = inputs.make_instance(n, m, 12)
    perm, d1, d2 = inputs.random_nodes(n, 60, seed=5, dmax=3)
    b1, b2 = orc.children_bounds_batch(p, perm, d1, d2, kind=orc.LB1 | orc.LB2 | orc.MINHT)
    c1, c2 = orc.children_bounds_batch(p, perm, d1, d2)
    for i in range(len(d1)):
        s1 = [int(x) for x in perm[i, :d1[i]]]
        s2 = [int(x) for x in perm[i, n - d2[i]:]]
        for j in perm[i, d1[i]:n - d2[i]]:
            j = int(j)
            f = orc.lb1(p, s1 + [j], s2, minht=True)
            b = orc.lb1(p, s1, [j] + s2, minht=True)
            assert (b1[i, 0, j], b1[i, 1, j]) == (f, b)
            # LB2 with the refinement: the larger of the refined LB1 and the pairs
            assert b2[i, 0, j] == max(c2[i, 0, j], f) and b2[i, 1, j] == max(c2[i, 1, j], b)


@pytest.mark.parametrize("seed", range(4))
def test_bounds_valid_sampled(seed):
    n, m = 8, 6
    p = inputs.make_instance(n, m, 50 + seed)
    perm, d1, d2 = inputs.random_nodes(n, 40, seed, dmax=4)
    for i in range(len(d1)):
        s1 = list(perm[i, :d1[i]])
        s2 = list(perm[i, n - d2[i]:])
        a = orc.lb1(p, s1, s2)
        b = orc.lb2(p, s1, s2)
        assert a <= b <= _completions_min(p, s1, s2)


def test_lb2_equals_max_over_pairs_of_bruteforce_relaxation():
    # LB2 = max over machine pairs of the optimum of the pair's two-machine
    # relaxation; the optimum is found here by trying every order of the
    # unscheduled jobs, so no Johnson order is involved.
    rng = np.random.default_rng(5)
    for seed in range(4):
        n, m = 7, 4
        p = inputs.make_instance(n, m, 200 + seed)
        jobs = rng.permutation(n)
        s1, s2 = list(jobs[:1]), list(jobs[5:])
        rest = [j for j in range(n) if j not in s1 and j not in s2]
        f, b = orc.front(p, s1), orc.back(p, s2)
        want = max(min(orc.pair_value(p, k, l, f, b, s) for s in itertools.permutations(rest))
                   for k in range(m) for l in range(k + 1, m))
        assert orc.lb2(p, s1, s2) == want


def _pair_list(m):
    return [(k, l) for k in range(m) for l in range(k + 1, m)]


def test_lb2_over_pair_subsets():
    # LB2 restricted to some machine pairs (the paper's LB2 uses between m and
    # m(m-1)/2 pairs) is max(LB1, optimum of each kept pair's two-machine
    # relaxation), the relaxation solved by trying every order of the
    # unscheduled jobs; all pairs in any order give the full LB2
    rng = np.random.default_rng(11)
    n, m = 7, 4
    P = m * (m - 1) // 2
    pairs = _pair_list(m)
    for seed in range(4):
        p = inputs.make_instance(n, m, 300 + seed)
        jobs = rng.permutation(n)
        d1, d2 = int(rng.integers(0, 2)), int(rng.integers(1, 3))
        perm = np.array(jobs, dtype=np.uint8)
        b1, b2full = orc.children_bounds_batch(p, perm[None], np.array([d1], np.uint8), np.array([d2], np.uint8))
        s1, s2 = list(perm[:d1]), list(perm[n - d2:])
        rest = [j for j in range(n) if j not in s1 and j not in s2]
        for subset in ([0], [P - 1], [2, 0], list(rng.permutation(P)[:3]), list(rng.permutation(P))):
            _, b2 = orc.children_bounds_batch(p, perm[None], np.array([d1], np.uint8),
                                              np.array([d2], np.uint8), pairs=subset)
            for d in (0, 1):
                for j in rest:
                    c1, c2 = (s1 + [j], s2) if d == 0 else (s1, [j] + s2)
                    others = [x for x in rest if x != j]
                    f, bk = orc.front(p, c1), orc.back(p, c2)
                    want = b1[0, d, j]
                    for q in subset:
                        k, l = pairs[q]
                        want = max(want, min(orc.pair_value(p, k, l, f, bk, list(o))
                                             for o in itertools.permutations(others)))
                    assert b2[0, d, j] == want, (subset, d, j)
                    assert b1[0, d, j] <= b2[0, d, j] <= b2full[0, d, j]
            if len(subset) == P:
                assert (b2 == b2full).all()


@pytest.mark.parametrize("seed", range(3))
def test_bb_with_adjacent_pairs_matches_brute_force(seed):
    # any valid bound keeps the search exact: LB2 over the m - 1 adjacent
    # machine pairs finds the brute-force optimum and explores a tree between
    # those of LB1 and of the full LB2
    n, m = 8, 4
    p = inputs.make_instance(n, m, 40 + seed)
    adjacent = [k * (2 * m - k - 1) // 2 for k in range(m - 1)]  # pair (k, k + 1)
    assert [_pair_list(m)[q] for q in adjacent] == [(k, k + 1) for k in range(m - 1)]
    cb, _ = orc.brute_force(p)
    r = orc.bb_solve(p, bound=orc.LB2, pairs=adjacent)
    assert r["cmax"] == cb and orc.makespan(p, r["perm"]) == cb
    t1 = orc.bb_solve(p, bound=orc.LB1, init_ub=cb)["decomposed"]
    ta = orc.bb_solve(p, bound=orc.LB2, init_ub=cb, pairs=adjacent)["decomposed"]
    t2 = orc.bb_solve(p, bound=orc.LB2, init_ub=cb)["decomposed"]
    assert t2 <= ta <= t1


@pytest.mark.parametrize("seed", range(5))
def test_leaf_bounds_are_exact(seed):
    n, m = 9, 5
    p = inputs.make_instance(n, m, seed)
    perm = np.random.default_rng(seed).permutation(n)
    c = orc.makespan(p, perm)
    for cut in range(n + 1):
        s1, s2 = list(perm[:cut]), list(perm[cut:])
        assert orc.lb1(p, s1, s2) == c
        assert orc.lb2(p, s1, s2) == c


@pytest.mark.parametrize("seed", range(5))
def test_two_machine_root_lb2_is_johnson_optimum(seed):
    p = inputs.make_instance(8, 2, 30 + seed)
    cj, _ = orc.johnson(p)
    cb, _ = orc.brute_force(p)
    assert orc.lb2(p, [], []) == cj == cb


def test_children_bounds_layout_matches_explicit_children():
    n, m = 7, 4
    p = inputs.make_instance(n, m, 11)
    perm = np.array([4, 0, 2, 6, 1, 3, 5], dtype=np.uint8)
    d1, d2 = 2, 1  # sigma1 = (4, 0), sigma2 = (5), unscheduled {2, 6, 1, 3}
    b1, b2 = orc.children_bounds(p, perm, d1, d2)
    for j in range(n):
        if j in (4, 0, 5):
            assert b1[0, j] == b1[1, j] == b2[0, j] == b2[1, j] == -1
            continue
        assert b1[0, j] == orc.lb1(p, [4, 0, j], [5])
        assert b1[1, j] == orc.lb1(p, [4, 0], [j, 5])
        assert b2[0, j] == orc.lb2(p, [4, 0, j], [5])
        assert b2[1, j] == orc.lb2(p, [4, 0], [j, 5])


def test_children_bounds_batch_matches_single():
    n, m = 10, 6
    p = inputs.make_instance(n, m, 3)
    perm, d1, d2 = inputs.random_nodes(n, 50, 9, dmax=5)
    o1, o2 = orc.children_bounds_batch(p, perm, d1, d2, threads=3)
    for i in range(50):
        a, b = orc.children_bounds(p, perm[i], d1[i], d2[i])
        assert (o1[i] == a).all() and (o2[i] == b).all()


# ---------------------------------------------------------------- MinMin ---

def test_minmin_worked_example():
    g = golden("minmin_example.json")
    n = 7
    lbf = np.full(n, -1)
    lbb = np.full(n, -1)
    jobs = [j - 1 for j in g["jobs_1based"]]
    lbf[jobs] = g["lb_forward"]
    lbb[jobs] = g["lb_backward"]
    d = orc.minmin(lbf, lbb, jobs)
    assert d == (orc.BWD if g["decision"] == "backward" else orc.FWD)
    ub = g["incumbent"]
    assert sum(v >= ub for v in g["lb_backward"]) == g["pruned_if_backward"]
    assert sum(v >= ub for v in g["lb_forward"]) == g["pruned_if_forward"]


def test_other_rules_on_the_worked_example():
    # Fig. 4's decomposition: backward leaves one child below the incumbent
    # (two pruned) and forward two (one pruned), so MinBranch also branches
    # backward; backward's bounds sum to 57 against forward's 53, so MinSum does too
    g = golden("minmin_example.json")
    n = 7
    lbf = np.full(n, -1)
    lbb = np.full(n, -1)
    jobs = [j - 1 for j in g["jobs_1based"]]
    lbf[jobs] = g["lb_forward"]
    lbb[jobs] = g["lb_backward"]
    ub = g["incumbent"]
    want = orc.BWD if g["decision"] == "backward" else orc.FWD
    for rule in (orc.MINMIN, orc.MINBRANCH, orc.MINSUM):
        assert orc.branch_rule(lbf, lbb, jobs, rule, cap=ub) == want


def test_branching_rules_disagree_by_hand():
    # hand-made bound vectors on which the rules part ways
    # MinMin: the minimum 16 occurs only backward -> forward.  MinBranch with
    # initial incumbent 18: two forward children below it, one backward -> backward.
    # MinSum: 64 forward against 66 backward -> backward.
    lbf, lbb = [17, 17, 30], [16, 25, 25]
    assert orc.branch_rule(lbf, lbb, [0, 1, 2], orc.MINMIN, cap=18) == orc.FWD
    assert orc.branch_rule(lbf, lbb, [0, 1, 2], orc.MINBRANCH, cap=18) == orc.BWD
    assert orc.branch_rule(lbf, lbb, [0, 1, 2], orc.MINSUM, cap=18) == orc.BWD
    # MinBranch backward (1 survivor of incumbent 20 against 2); MinSum forward (111 > 72)
    lbf, lbb = [10, 11, 90], [12, 30, 30]
    assert orc.branch_rule(lbf, lbb, [0, 1, 2], orc.MINBRANCH, cap=20) == orc.BWD
    assert orc.branch_rule(lbf, lbb, [0, 1, 2], orc.MINSUM, cap=20) == orc.FWD
    # MinBranch tie (one survivor each) -> larger sum (40 > 32) -> forward
    assert orc.branch_rule([10, 30], [12, 20], [0, 1], orc.MINBRANCH, cap=15) == orc.FWD
    # equal sums -> forward under both
    assert orc.branch_rule([5, 8], [6, 7], [0, 1], orc.MINSUM) == orc.FWD
    assert orc.branch_rule([5, 8], [6, 7], [0, 1], orc.MINBRANCH, cap=7) == orc.FWD
    # only unscheduled jobs count
    assert orc.branch_rule([1, 50, 50], [1, 40, 40], [1, 2], orc.MINSUM) == orc.FWD


def test_minmin_tie_rules():
    # equal counts of the minimum -> larger sum wins; equal sums -> forward
    assert orc.minmin([5, 9], [5, 7], [0, 1]) == orc.FWD
    assert orc.minmin([5, 7], [5, 9], [0, 1]) == orc.BWD
    assert orc.minmin([5, 8], [5, 8], [0, 1]) == orc.FWD
    # capped values: both sets above the cap look identical
    assert orc.minmin([20, 30], [25, 40], [0, 1], cap=10) == orc.FWD


@pytest.mark.parametrize("capped", [False, True])
def test_minmin_picks_a_fully_pruned_direction(capped):
    # Brute force over small bound vectors: when every child of one direction
    # is at or above the incumbent, MinMin's choice leaves no child below it
    # (the early exit of the LB2 sweep relies on this).  A plausible slip in
    # the rule (counting the more frequent minimum, or the smaller sum first)
    # fails here.
    rng = np.random.default_rng(7 + capped)
    ub = 10
    for _ in range(4000):
        u = int(rng.integers(1, 5))
        jobs = list(range(u))
        full = rng.integers(ub, ub + 4, size=u)      # one direction entirely >= ub
        other = rng.integers(ub - 3, ub + 3, size=u)  # the other one mixed
        for lbf, lbb in ((full, other), (other, full)):
            d = orc.minmin(lbf, lbb, jobs, cap=ub if capped else orc.INT32_MAX)
            chosen = lbf if d == orc.FWD else lbb
            assert all(v >= ub for v in chosen), (lbf, lbb, d)


def test_minbranch_picks_a_fully_pruned_direction():
    # the same dead-end property for MinBranch (counting against the initial
    # incumbent): a direction with every child at or above it has no survivor,
    # so MinBranch picks it unless the other has none either, and then no child
    # of either direction survives (the early exit stays exact under MinBranch)
    rng = np.random.default_rng(11)
    ub = 10
    for _ in range(4000):
        u = int(rng.integers(1, 5))
        jobs = list(range(u))
        full = rng.integers(ub, ub + 4, size=u)
        other = rng.integers(ub - 3, ub + 3, size=u)
        for lbf, lbb in ((full, other), (other, full)):
            d = orc.branch_rule(lbf, lbb, jobs, orc.MINBRANCH, cap=ub)
            chosen = lbf if d == orc.FWD else lbb
            assert all(v >= ub for v in chosen), (lbf, lbb, d)


def test_minsum_may_branch_away_from_a_fully_pruned_direction():
    # why the early exit is refused with MinSum: forward is entirely at or
    # above the incumbent 10, yet backward's larger sum (39 > 20) wins, and
    # backward keeps a child (9) below the incumbent; an early exit would have
    # replaced backward's LB2 by lower LB1 values and could flip the decision
    assert orc.branch_rule([10, 10], [9, 30], [0, 1], orc.MINSUM, cap=10) == orc.BWD
    assert orc.branch_rule([10, 10], [9, 30], [0, 1], orc.MINBRANCH, cap=10) == orc.FWD


# ---------------------------------------------------------------- search ---

@pytest.mark.parametrize("seed", range(1, 11))
def test_bb_lb1_neh_matches_brute_force_n10_m5(seed):
    # 10 jobs, 5 machines, LB1, incumbent initialised from NEH
    p = inputs.make_instance(10, 5, seed)
    r = orc.bb_solve(p, bound=orc.LB1)
    cb, _ = orc.brute_force(p)
    assert r["outcome"] == orc.OPTIMAL
    assert r["cmax"] == cb
    assert orc.makespan(p, r["perm"]) == cb
    assert sorted(r["perm"]) == list(range(10))


@pytest.mark.parametrize("seed", range(4))
def test_bb_lb2_matches_brute_force(seed):
    p = inputs.make_instance(8, 4, 40 + seed)
    r = orc.bb_solve(p, bound=orc.LB2)
    cb, _ = orc.brute_force(p)
    assert r["cmax"] == cb and orc.makespan(p, r["perm"]) == cb


def _py_rule(rule, lbf, lbb, un, ub):
    """MinBranch / MinSum decisions restated from their definitions, on Python lists."""
    f = [int(lbf[j]) for j in un]
    b = [int(lbb[j]) for j in un]
    if rule == orc.MINBRANCH:
        kf, kb = sum(v < ub for v in f), sum(v < ub for v in b)
        if kf != kb:
            return orc.FWD if kf < kb else orc.BWD
    return orc.BWD if sum(b) > sum(f) else orc.FWD


def _critical_tree_bfs(p, bound, ub, capped=False, rule=None, minht=False):
    """Count decomposed nodes level by level (breadth first), independent of the DFS."""
    n = p.shape[0]
    kind = (orc.LB1 if bound == orc.LB1 else orc.LB2) | (orc.MINHT if minht else 0)
    level = [(list(range(n)), 0, 0)]
    decomposed = bounded = 0
    while level:
        nxt = []
        for perm, d1, d2 in level:
            decomposed += 1
            u = n - d1 - d2
            bounded += 2 * u
            b1, b2 = orc.children_bounds(p, np.array(perm, dtype=np.uint8), d1, d2, kind)
            lb = b1 if bound == orc.LB1 else b2
            un = perm[d1:n - d2]
            if rule is None:
                d = orc.minmin(lb[0], lb[1], un, cap=ub if capped else orc.INT32_MAX)
            else:
                d = _py_rule(rule, lb[0], lb[1], un, ub)
            if u == 1:
                continue
            for j in un:
                if lb[d, j] >= ub:
                    continue
                rest = [x for x in un if x != j]
                if d == orc.FWD:
                    nxt.append((perm[:d1] + [j] + rest + perm[n - d2:], d1 + 1, d2))
                else:
                    nxt.append((perm[:d1] + rest + [j] + perm[n - d2:], d1, d2 + 1))
        level = nxt
    return decomposed, bounded


@pytest.mark.parametrize("bound,seed", [(orc.LB1, 1), (orc.LB1, 2), (orc.LB2, 3), (orc.LB2, 4)])
def test_proof_mode_node_count_matches_breadth_first_enumeration(bound, seed):
    p = inputs.make_instance(8, 4, seed)
    opt, _ = orc.brute_force(p)
    r = orc.bb_solve(p, bound=bound, init_ub=opt)
    assert r["outcome"] == orc.PROVEN_NO_BETTER
    dec, bnd = _critical_tree_bfs(p, bound, opt)
    assert r["decomposed"] == dec and r["bounded"] == bnd
    rc = orc.bb_solve(p, bound=bound, init_ub=opt, capped=True)
    dec_c, _ = _critical_tree_bfs(p, bound, opt, capped=True)
    assert rc["decomposed"] == dec_c


@pytest.mark.parametrize("bound,seed", [(orc.LB1, 5), (orc.LB2, 6), (orc.LB2, 7)])
@pytest.mark.parametrize("rule", [orc.MINBRANCH, orc.MINSUM])
def test_other_branching_rules_proof_counts(rule, bound, seed):
    # the DFS under MinBranch / MinSum explores exactly the tree that a
    # breadth-first enumeration with the rules restated in Python gives
    p = inputs.make_instance(8, 4, seed)
    opt, _ = orc.brute_force(p)
    r = orc.bb_solve(p, bound=bound, init_ub=opt, branching=rule)
    assert r["outcome"] == orc.PROVEN_NO_BETTER
    dec, bnd = _critical_tree_bfs(p, bound, opt, rule=rule)
    assert r["decomposed"] == dec and r["bounded"] == bnd


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("rule", [orc.MINMIN, orc.MINMIN_CAPPED, orc.MINBRANCH, orc.MINSUM])
def test_every_branching_rule_finds_the_brute_force_optimum(rule, seed):
    n, m = 8, 4
    p = inputs.make_instance(n, m, 60 + seed)
    cb, _ = orc.brute_force(p)
    for bound in (orc.LB1, orc.LB2):
        r = orc.bb_solve(p, bound=bound, branching=rule)
        assert r["cmax"] == cb and orc.makespan(p, r["perm"]) == cb


@pytest.mark.parametrize("bound,seed", [(orc.LB1, 13), (orc.LB1, 20), (orc.LB1, 23), (orc.LB2, 11)])
def test_minht_proof_counts_and_optimum(bound, seed):
    # with the refinement the DFS reaches the brute-force optimum and its
    # proof tree is the breadth-first enumeration's with the refined bounds
    # (LB1 trees of these seeds differ from the plain ones: 85 -> 57,
    # 102 -> 103, 72 -> 73 nodes; full-pair LB2 dominates the refined LB1
    # on 8 x 4 instances and keeps its trees)
    p = inputs.make_instance(8, 4, seed)
    opt, _ = orc.brute_force(p)
    r = orc.bb_solve(p, bound=bound, minht=True)
    assert r["cmax"] == opt and orc.makespan(p, r["perm"]) == opt
    q = orc.bb_solve(p, bound=bound, init_ub=opt, minht=True)
    dec, bnd = _critical_tree_bfs(p, bound, opt, minht=True)
    assert q["decomposed"] == dec and q["bounded"] == bnd


def test_bb_node_limit():
    p = inputs.make_instance(12, 5, 1)
    r = orc.bb_solve(p, bound=orc.LB1, init_ub=1, node_limit=0)
    assert r["outcome"] == orc.PROVEN_NO_BETTER and r["decomposed"] == 1  # root only
    r = orc.bb_solve(p, bound=orc.LB1, init_ub=10**6, node_limit=50)
    assert r["outcome"] == orc.LIMIT_NODES and r["decomposed"] == 50


# ---------------------------------------------------------------- NEH ------

def test_neh_hand_example():
    g = golden("neh_hand_example.json")
    p = np.array(g["p"])
    c, perm = orc.neh(p)
    assert c == g["neh_cmax"] and list(perm) == g["neh_perm"]
    assert orc.brute_force(p)[0] == g["optimum"]
    assert orc.makespan(p, g["makespan_01_of_first_two_jobs"]["perm"] + [2]) >= 12


@pytest.mark.parametrize("seed", range(5))
def test_neh_is_a_valid_upper_bound(seed):
    p = inputs.make_instance(8, 5, seed)
    c, perm = orc.neh(p)
    assert sorted(perm) == list(range(8))
    assert orc.makespan(p, perm) == c >= orc.brute_force(p)[0]


# ---------------------------------------------------------------- IVM / intervals

def test_ivm_decode_example():
    g = golden("ivm_decode_example.json")
    jobs = [j - 1 for j in g["jobs_1based"]]
    dirs = [orc.FWD if d == "forward" else orc.BWD for d in g["dirs"]]
    s1, s2 = orc.ivm_decode(jobs, dirs)
    assert [j + 1 for j in s1] == g["sigma1_1based"]
    assert [j + 1 for j in s2] == g["sigma2_1based"]
    un = sorted(set(range(g["n"])) - set(s1) - set(s2))
    assert [j + 1 for j in un] == g["unscheduled_1based"]


def test_factoradic_counter_n5():
    g = golden("factoradic_examples.json")
    seen = [list(orc.factoradic_from_decimal(5, x)) for x in range(math.factorial(5))]
    assert len(seen) == g["n5_count"]
    assert seen[0] == g["n5_first"] and seen[1] == g["n5_second"] and seen[2] == g["n5_third"]
    assert seen[-1] == g["n5_last"]
    # every digit vector is valid (digit i has radix n - i) and they are distinct and increasing
    for v in seen:
        assert all(0 <= v[i] < 5 - i for i in range(5))
    assert seen == sorted(seen) and len({tuple(v) for v in seen}) == 120


def test_factoradic_work_units_n4():
    g = golden("factoradic_examples.json")
    for dec, digits in g["n4_decimal_to_factoradic"].items():
        assert list(orc.factoradic_from_decimal(4, int(dec))) == digits
        assert orc.factoradic_to_decimal(digits) == int(dec)
    units = g["n4_units_decimal"]
    assert units[0][0] == 0 and units[-1][1] == math.factorial(4)


@pytest.mark.parametrize("n", range(1, 9))
def test_factoradic_round_trip(n):
    for x in range(math.factorial(n)):
        assert orc.factoradic_to_decimal(orc.factoradic_from_decimal(n, x)) == x


def test_factoradic_is_lexicographic_leaf_numbering():
    # digit i = rank of the job picked at level i among the remaining jobs in
    # ascending order; decimal order = lexicographic order of the permutations
    n = 5
    for x, perm in enumerate(itertools.permutations(range(n))):
        rest = list(range(n))
        digits = []
        for j in perm:
            digits.append(rest.index(j))
            rest.remove(j)
        assert orc.factoradic_to_decimal(digits) == x


def test_steal_midpoint():
    assert orc.steal_midpoint(0, 24) == 12
    assert orc.steal_midpoint(9, 15) == 12
    assert orc.steal_midpoint(16, 24) == 20
    assert orc.steal_midpoint(5, 6) == 5
    big = math.factorial(20)
    assert orc.steal_midpoint(0, big) == big // 2
