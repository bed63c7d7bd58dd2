"""pfsp_solve_noalloc agrees with pfsp_solve.

pfsp_solve_noalloc exists for programs that may not allocate device memory
when they solve: services that reserve all their memory at start-up,
applications whose device memory is owned by another allocator, and callers
that cannot accept the device synchronisation an allocation brings.  It keeps
its scratch in one static array per device instead of calling cudaMalloc.

The test calls it twice in a row through the C ABI, on two different
instances, and compares each result with the allocating entry point: the same
optimum and outcome in finding mode, and in proof mode the same exact
decomposed-node and bounded-children counts.  The second call also checks that
the scratch left behind by the first call does not leak into the next one.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2012_09511_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import pfsp
    return pfsp


def _makespan(p, perm):
    m = p.shape[1]
    c = np.zeros(m, dtype=np.int64)
    for j in perm:
        prev = 0
        for k in range(m):
            c[k] = max(c[k], prev) + p[j, k]
            prev = c[k]
    return int(c[-1])


def test_noalloc_matches_allocating_solve_twice(pf):
    # first call: finding mode from NEH, LB1
    p1 = inputs.make_instance(10, 5, 3)
    ref1 = pf.pfsp_solve(pf.pfsp_load_instance(p1), bound=pf.PFSP_LB1)
    got1 = pf.pfsp_solve_noalloc(p1, bound=pf.PFSP_LB1)
    assert (got1["cmax"], got1["outcome"]) == (ref1["cmax"], ref1["outcome"])
    assert sorted(got1["perm"].tolist()) == list(range(10))
    assert _makespan(p1, got1["perm"]) == got1["cmax"]

    # second call, another shape: proof mode at the optimum, LB2; the tree is
    # fixed, so the counts must agree exactly
    p2 = inputs.make_instance(12, 10, 17)
    inst2 = pf.pfsp_load_instance(p2)
    opt = pf.pfsp_solve(inst2, bound=pf.PFSP_LB2)["cmax"]
    ref2 = pf.pfsp_solve(inst2, bound=pf.PFSP_LB2, init_ub=opt)
    got2 = pf.pfsp_solve_noalloc(p2, bound=pf.PFSP_LB2, init_ub=opt)
    assert got2["outcome"] == ref2["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert got2["cmax"] == ref2["cmax"] == opt
    assert (got2["decomposed"], got2["bounded_children"]) == (ref2["decomposed"], ref2["bounded_children"])
    assert got2["decomposed"] > 1


def test_noalloc_large_n_shrinks_pool(pf):
    # at n = 50 the 12-warp-per-SM pool needs about 23 MB: the call must shrink
    # the pool (down to one explorer per SM if needed) and still solve
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    p = inputs.make_instance(50, 5, 101)
    got = pf.pfsp_solve_noalloc(p, bound=pf.PFSP_LB1, node_limit=20000)
    assert got["outcome"] in (pf.PFSP_OPTIMAL, pf.PFSP_LIMIT_NODES)
    assert sorted(got["perm"].tolist()) == list(range(50))
    assert _makespan(p, got["perm"]) == got["cmax"]
    # the pool holds at least one explorer per SM and fits the 8 MiB array
    # (rows of n x n jobs and bounds, 5 bytes a cell, plus 209 bytes of state)
    assert nsm <= got["explorers"]
    assert got["explorers"] * (50 * 50 * 5 + 209) < 8 << 20
    # the search starts from NEH, so its incumbent is never worse (oracle's NEH)
    import oracle
    assert got["cmax"] <= oracle.neh(p)[0]


def test_noalloc_largest_n_and_rejections(pf):
    # n = 64, the library's largest instance, is accepted
    p = inputs.make_instance(64, 5, 7)
    got = pf.pfsp_solve_noalloc(p, bound=pf.PFSP_LB1, node_limit=5000)
    assert sorted(got["perm"].tolist()) == list(range(64))
    assert _makespan(p, got["perm"]) == got["cmax"]
    # LB2 tables that exceed shared memory (m = 64: 2,016 pairs) are refused
    # with PFSP_ERR_UNSUPPORTED before any device work
    with pytest.raises(pf.PfspError) as e:
        pf.pfsp_solve_noalloc(inputs.make_instance(20, 64, 1), bound=pf.PFSP_LB2)
    assert e.value.code == pf.PFSP_ERR_UNSUPPORTED
    # a third solve after the refusal still agrees with the allocating one
    p3 = inputs.make_instance(10, 5, 4)
    ref = pf.pfsp_solve(pf.pfsp_load_instance(p3), bound=pf.PFSP_LB1)
    got3 = pf.pfsp_solve_noalloc(p3, bound=pf.PFSP_LB1)
    assert (got3["cmax"], got3["outcome"]) == (ref["cmax"], ref["outcome"])
