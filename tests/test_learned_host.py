"""Host logic of the learned solver's workflow (CPU, no GPU): the root's
children that learned.order_pairs scores, in the node layout of
pfsp_bound_batch, must be the root's 2n children as the oracle defines them
(Section 2.3: a child schedules one more job at the front or at the back)."""
import numpy as np

import oracle as orc
from paper_2012_09511_gb300 import inputs, learned


def test_root_children_are_the_oracle_children_of_the_root():
    n, m = 7, 5
    p = inputs.make_instance(n, m, 3)
    perm, d1, d2 = learned.root_children(n)
    assert perm.shape == (2 * n, n) and d1.shape == d2.shape == (2 * n,)
    # every row is a permutation with one scheduled job: first (forward) or last (backward)
    for r in range(2 * n):
        assert sorted(perm[r].tolist()) == list(range(n))
        assert (d1[r], d2[r]) == ((1, 0) if r < n else (0, 1))
    assert (perm[:n, 0] == np.arange(n)).all() and (perm[n:, -1] == np.arange(n)).all()
    # the bounds of these nodes are the oracle's bounds of the root's children
    lb1, lb2 = orc.children_bounds(p, np.arange(n, dtype=np.uint8), 0, 0)
    for j in range(n):
        assert orc.lb1(p, [j], []) == lb1[0, j] and orc.lb2(p, [j], []) == lb2[0, j]
        assert orc.lb1(p, [], [j]) == lb1[1, j] and orc.lb2(p, [], [j]) == lb2[1, j]
        # the row's own partial schedule is the one the child stands for
        assert orc.lb2(p, list(perm[j, :1]), []) == lb2[0, j]
        assert orc.lb2(p, [], list(perm[n + j, -1:])) == lb2[1, j]


class _Flags:
    PFSP_EARLY_EXIT, PFSP_EARLY_EXIT_SLOTS, PFSP_EARLY_EXIT_CHILDREN = 4, 8, 16


def test_slot_checks_from_four_slots():
    # the learned solver checks after every 32-pair slot from four slots on
    # (more than 96 pairs: m >= 15), where the network's order can act
    assert [m for m in range(2, 33) if learned.slot_checks_for(m)] == list(range(15, 33))
    f = _Flags()
    assert learned.learned_options(f, m=20)["learned"] == 4 | 8 | 16
    assert learned.learned_options(f, m=10)["learned"] == 4 | 16
    assert learned.learned_options(f)["learned"] == 4 | 16
    assert learned.learned_options(f, slot_checks=True, m=10)["learned"] == 4 | 8 | 16
    assert learned.learned_options(f, slot_checks=False, m=20)["learned"] == 4 | 16
