"""Parity of the batched explorer pool (pfsp_solve_batch) with the CPU oracle.

Every instance of a batch must get the oracle's optimum, a valid permutation
reaching it, and in proof mode (every incumbent at its optimum) the summed
decomposed-node count must equal the sum of the oracle's fixed-tree counts.
The full workload is 256 instances of uneven shape (n in 12..20, m in
{5, 10, 20}) solved by one persistent launch from a CUDA graph; its optima come
from tests/golden/batch256_lb2.json, written by the oracle-only script beside
it (instances the oracle could not finish are reported, not compared).
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
from paper_2012_09511_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch256_lb2.json")


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import pfsp
    return pfsp


def _small_batch(count=24):
    shapes = [(8 + (i % 5), (5, 10, 20)[i % 3]) for i in range(count)]
    return [inputs.make_instance(n, m, 500 + i) for i, (n, m) in enumerate(shapes)]


def _check_perm(p, row, cmax):
    n = p.shape[0]
    perm = row[:n]
    assert sorted(perm.tolist()) == list(range(n))
    assert (row[n:] == -1).all()
    assert orc.makespan(p, perm) == cmax


@pytest.mark.parametrize("bound", [1, 2])
def test_small_uneven_batch_optima(pf, bound):
    ps = _small_batch()
    insts = [pf.pfsp_load_instance(p) for p in ps]
    r = pf.pfsp_solve_batch(insts, bound=bound)
    for i, p in enumerate(ps):
        want = orc.bb_solve(p, bound=bound)["cmax"]
        assert r["outcomes"][i] == pf.PFSP_OPTIMAL
        assert r["cmax"][i] == want, (i, p.shape)
        _check_perm(p, r["perms"][i], want)


@pytest.mark.parametrize("rule", ["MINMIN", "MINBRANCH", "MINSUM"])
def test_small_batch_proof_mode_counts(pf, rule):
    ps = _small_batch(18)
    opts = [orc.bb_solve(p, bound=2)["cmax"] for p in ps]
    br = getattr(orc, rule)
    want = sum(orc.bb_solve(p, bound=2, init_ub=o, branching=br)["decomposed"] for p, o in zip(ps, opts))
    insts = [pf.pfsp_load_instance(p) for p in ps]
    r = pf.pfsp_solve_batch(insts, bound=2, init_ubs=opts, branching=getattr(pf, "PFSP_" + rule))
    assert (r["outcomes"] == pf.PFSP_PROVEN_NO_BETTER).all()
    assert (r["cmax"] == np.array(opts)).all()
    assert r["stats"]["decomposed"] == want
    assert (r["perms"] == -1).all()


def test_batch_agrees_with_single_solves(pf):
    ps = _small_batch(12)
    insts = [pf.pfsp_load_instance(p) for p in ps]
    r = pf.pfsp_solve_batch(insts, bound=2, warps_per_sm=4)
    for i, inst in enumerate(insts):
        s = pf.pfsp_solve(inst, bound=2)
        assert s["cmax"] == r["cmax"][i]


def test_empty_and_invalid_batches(pf):
    r = pf.pfsp_solve_batch([], bound=2)
    assert len(r["cmax"]) == 0
    inst = pf.pfsp_load_instance(inputs.make_instance(8, 5, 1))
    with pytest.raises(pf.PfspError):
        pf.pfsp_solve_batch([inst], bound=7)


@pytest.mark.parametrize("per_sm,slot", [(12, 4), (8, 4), (12, 6), (4, 4)])
def test_instance_slots_and_explorers_per_sm(pf, per_sm, slot):
    # explorers per SM and explorers per instance slot are honoured: the pool
    # has SMs x per_sm explorers, and the optima do not depend on the shape
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ps = _small_batch(12)
    insts = [pf.pfsp_load_instance(p) for p in ps]
    r = pf.pfsp_solve_batch(insts, bound=2, warps_per_sm=per_sm, slot_warps=slot)
    assert r["stats"]["explorers"] == nsm * (per_sm // slot) * slot
    for i, p in enumerate(ps):
        assert r["cmax"][i] == orc.bb_solve(p, bound=2)["cmax"]


def test_autotuner_returns_usable_options(pf):
    ps = _small_batch(16)
    insts = [pf.pfsp_load_instance(p) for p in ps]
    best = pf.pfsp_autotune_batch(insts, pf.pfsp_default_options(bound=2), sample=8)
    assert best.warps_per_sm in (8, 12) and best.slot_warps in (4, 6, 12) and best.slot_warps <= best.warps_per_sm
    assert best.check_every in (8, 32) and best.min_steal in (2.0, 40320.0)
    r = pf.pfsp_solve_batch(insts, best)
    for i, p in enumerate(ps):
        assert r["cmax"][i] == orc.bb_solve(p, bound=2)["cmax"]


def test_batch256_uneven_optima(pf):
    if not os.path.exists(GOLDEN):
        pytest.skip("oracle optima not generated (tests/golden/make_batch_golden.py)")
    with open(GOLDEN) as f:
        g = {r["i"]: r for r in json.load(f)["results"]}
    ps, shapes = [], []
    for i in range(256):
        n, m = inputs.batch_instance_shape(i)
        shapes.append((n, m))
        ps.append(inputs.make_instance(n, m, 1000 + i))
    insts = [pf.pfsp_load_instance(p) for p in ps]
    r = pf.pfsp_solve_batch(insts, bound=2)
    assert (r["outcomes"] == pf.PFSP_OPTIMAL).all()
    verified = 0
    for i, p in enumerate(ps):
        _check_perm(p, r["perms"][i], r["cmax"][i])
        if i in g and "optimum" in g[i]:
            assert r["cmax"][i] == g[i]["optimum"], (i, shapes[i])
            verified += 1
    # every instance has a record; those without an optimum say why (the
    # oracle's node budget), and they are listed here by id
    assert sorted(g) == list(range(256))
    unverified = [i for i in range(256) if "optimum" not in g[i]]
    assert all("unverified" in g[i] for i in unverified)
    assert verified == 256 - len(unverified), (verified, unverified)
