"""The roofline numerators bench.py reports, checked on the CPU.

algorithmic_ops counts what the kernel's O(P u) composition does per parent;
child_by_child_ops what the paper's recurrence does child by child.  Both are
checked against sums written out node by node for a few depth pairs, and the
ratio between them at the benchmark's depth mix is pinned.
"""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_op_counts_node_by_node():
    b = _bench()
    n, m = 20, 20
    P = m * (m - 1) // 2
    d1 = np.array([0, 3, 10, 20, 19], dtype=np.uint8)
    d2 = np.array([0, 5, 10, 0, 0], dtype=np.uint8)
    alg = cbc = 0
    for a, c in zip(d1.tolist(), d2.tolist()):
        u = n - a - c
        # wavefronts 2 per cell; LB1 6 per child and machine over 2u children;
        # LB2 13 per (pair, unscheduled job)
        alg += 2 * m * (a + c) + 2 * u * m * 6 + P * u * 13
        # child by child: LB2 4 per (child, pair, job of the child); LB1 4m per
        # child; the parent's wavefronts 2 per cell
        cbc += 4 * 2 * P * u * max(u - 1, 0) + 4 * m * 2 * u + 2 * m * (a + c)
    assert b.algorithmic_ops(n, m, d1, d2) == alg
    assert b.child_by_child_ops(n, m, d1, d2) == cbc


def test_benchmark_depth_mix_ratio():
    # at the benchmark's depth mix (d1, d2 uniform in 0..10) the child-by-child
    # count is about 6.1 times the composition's
    b = _bench()
    from paper_2012_09511_gb300 import inputs
    perm, d1, d2 = inputs.random_nodes(20, 200000, seed=2020)
    r = b.child_by_child_ops(20, 20, d1, d2) / b.algorithmic_ops(20, 20, d1, d2)
    assert 6.0 < r < 6.3
