"""Host heuristic threads' search (Section 4.2): the iterated greedy of
pfsp_iterated_greedy, checked on the CPU against the oracle.

Its results are pinned by what the mathematics fixes: the schedule is a
permutation whose makespan (oracle, Eq. 1) is the reported value; that value is
never below the brute-force or branch-and-bound optimum, never above the NEH
schedule it starts from, and reaches the brute-force optimum on small
instances.  Host code only: these tests need no GPU.
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
from paper_2012_09511_gb300 import inputs


@pytest.fixture(scope="module")
def pf():
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import pfsp
    return pfsp


def _valid(p, perm, c):
    assert sorted(perm.tolist()) == list(range(p.shape[0]))
    assert orc.makespan(p, perm) == c


@pytest.mark.parametrize("seed", range(6))
def test_reaches_brute_force_optimum_on_small_instances(pf, seed):
    p = inputs.make_instance(8, 4, 100 + seed)
    opt, _ = orc.brute_force(p)
    c, perm = pf.pfsp_iterated_greedy(p, 200, seed=seed)
    _valid(p, perm, c)
    assert c == opt


@pytest.mark.parametrize("seed", [1, 3, 5, 7])
def test_bounded_by_neh_and_the_optimum_20x10(pf, seed):
    with open(os.path.join(os.path.dirname(__file__), "golden", "solve_20x10_lb2.json")) as f:
        opt = {r["seed"]: r["optimum"] for r in json.load(f)["results"]}[seed]
    p = inputs.make_instance(20, 10, seed)
    neh_c, _ = orc.neh(p)
    c, perm = pf.pfsp_iterated_greedy(p, 300, seed=seed)
    _valid(p, perm, c)
    assert opt <= c <= neh_c
    assert c <= opt * 1.02  # the iterated greedy's usual quality on such instances


def test_start_schedule_and_determinism(pf):
    p = inputs.make_instance(15, 5, 9)
    start = np.arange(15, dtype=np.int32)[::-1].copy()
    c0 = orc.makespan(p, start)
    c, perm = pf.pfsp_iterated_greedy(p, 0, seed=4, start=start)  # local search only
    _valid(p, perm, c)
    assert c <= c0
    a = pf.pfsp_iterated_greedy(p, 50, seed=11, start=start)
    b = pf.pfsp_iterated_greedy(p, 50, seed=11, start=start)
    assert a[0] == b[0] and (a[1] == b[1]).all()
    assert a[0] <= c


def test_degenerate_shapes(pf):
    # one job; one machine (every order has the total work as makespan)
    p1 = np.array([[3, 4, 5]], dtype=np.int32)
    c, perm = pf.pfsp_iterated_greedy(p1, 10)
    assert c == 12 and perm.tolist() == [0]
    p2 = inputs.make_instance(9, 1, 2)
    c, perm = pf.pfsp_iterated_greedy(p2, 10)
    _valid(p2, perm, c)
    assert c == int(p2.sum())


def test_invalid_arguments(pf):
    p = inputs.make_instance(6, 3, 1)
    for kw in (dict(start=np.array([0, 1, 2, 3, 4, 4], dtype=np.int32)),
               dict(start=np.array([0, 1, 2, 3, 4, 9], dtype=np.int32))):
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_iterated_greedy(p, 5, **kw)
        assert e.value.code == pf.PFSP_ERR_INVALID
    with pytest.raises(pf.PfspError):
        pf.pfsp_iterated_greedy(p, -1)
    bad = p.copy()
    bad[0, 0] = -1
    with pytest.raises(pf.PfspError):
        pf.pfsp_iterated_greedy(bad, 5)


def _best_completion(p, prefix, suffix):
    import itertools
    n = p.shape[0]
    rest = [j for j in range(n) if j not in prefix and j not in suffix]
    return min(orc.makespan(p, list(prefix) + list(mid) + list(suffix)) for mid in itertools.permutations(rest))


@pytest.mark.parametrize("seed", range(4))
def test_beam_search_wide_enough_is_exhaustive(pf, seed):
    # a width of at least the number of partial schedules of every level keeps
    # them all: the beam search is then an enumeration and returns the optimum
    n, m = 7, 4
    p = inputs.make_instance(n, m, 200 + seed)
    opt, _ = orc.brute_force(p)
    c, perm = pf.pfsp_beam_search(p, 5040)
    _valid(p, perm, c)
    assert c == opt


@pytest.mark.parametrize("prefix,suffix", [([3], [5]), ([0, 6], []), ([], [1, 2]), ([4, 2, 0], [6, 1])])
def test_beam_search_keeps_the_node(pf, prefix, suffix):
    n, m = 8, 5
    p = inputs.make_instance(n, m, 31)
    best = _best_completion(p, prefix, suffix)
    for width in (1, 3, 40320):
        c, perm = pf.pfsp_beam_search(p, width, prefix=prefix, suffix=suffix)
        _valid(p, perm, c)
        assert perm[:len(prefix)].tolist() == prefix
        assert perm[n - len(suffix):].tolist() == suffix
        # never below the best completion, and the bound of the node is below both
        assert c >= best >= orc.lb1(p, prefix, suffix)
        if width == 40320:
            assert c == best


def test_beam_search_width_one_is_the_lb1_greedy_dive(pf):
    # width 1: at each level the extension of least LB1 (ties: smaller front sum)
    n, m = 9, 4
    p = inputs.make_instance(n, m, 17)
    c, perm = pf.pfsp_beam_search(p, 1)
    seq = []
    for _ in range(n):
        cand = []
        for j in range(n):
            if j in seq:
                continue
            lb = orc.lb1(p, seq + [j], [])
            fs = int(orc.completion(p, seq + [j]).sum())
            cand.append((lb, fs, j))
        seq.append(min(cand)[2])
    assert perm.tolist() == seq and c == orc.makespan(p, seq)


def test_beam_search_invalid_arguments(pf):
    p = inputs.make_instance(6, 3, 1)
    for kw in (dict(prefix=[0], suffix=[0]), dict(prefix=[9]), dict(prefix=[0, 1, 2, 3], suffix=[4, 5, 1])):
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_beam_search(p, 4, **kw)
        assert e.value.code == pf.PFSP_ERR_INVALID
    with pytest.raises(pf.PfspError):
        pf.pfsp_beam_search(p, 0)
