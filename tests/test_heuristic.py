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
