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
