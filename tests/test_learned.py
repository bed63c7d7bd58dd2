"""The learned ordering (network-ordered LB2 slots and rows, early exit).

* Training rows built on the GPU carry the oracle's features (per-machine
  front, back and remaining work over the mean machine load) and targets
  (pairs whose two-machine term is a child's LB2 above its LB1; the child of
  least LB2 per direction).
* The solver's traced nodes are valid nodes of the instance.
* Exactness: with any network the optimum is unchanged, and in proof mode
  capped MinMin with early exit and learned orders explores exactly the tree
  of plain capped MinMin (the oracle's capped count).  Early exit alone, with
  any pair order, keeps the oracle's counts under either MinMin rule.
* The pair order changes no bound and no training row; the learned order
  ranks the pairs by the network's mean pair probability.
* Training on the solver's own traces lowers the loss and predicts the pair
  targets better than the best constant per pair (what the network adds).
"""
import numpy as np
import pytest

import oracle as orc
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


def _pairs(m):
    return [(k, l) for k in range(m) for l in range(k + 1, m)]


def test_training_rows_match_oracle(pf):
    n, m = 8, 5
    p = inputs.make_instance(n, m, 12)
    scale = p.sum() / m
    perm, d1, d2 = inputs.random_nodes(n, 40, seed=3, dmax=4)
    inst = pf.pfsp_load_instance(p)
    mlp = pf.pfsp_mlp_create(m, seed=1)
    X, T, M = pf.pfsp_mlp_rows(inst, mlp, perm, d1, d2)
    rows = 1 + 2 * n
    pairs = _pairs(m)
    for i in range(len(d1)):
        s1, s2 = list(perm[i, :d1[i]]), list(perm[i, n - d2[i]:])
        un = [j for j in range(n) if j not in s1 and j not in s2]
        base = i * rows
        want = np.concatenate([orc.front(p, s1), orc.back(p, s2), orc.remain(p, un)]) / scale
        assert np.allclose(X[base, :3 * m], want, rtol=1e-6)
        b1, b2 = orc.children_bounds(p, perm[i], d1[i], d2[i])
        hits = np.zeros(len(pairs))
        for d in (0, 1):
            for j in un:
                c1, c2 = (s1 + [j], s2) if d == 0 else (s1, [j] + s2)
                r = base + 1 + d * n + j
                rest = [x for x in un if x != j]
                wf = np.concatenate([orc.front(p, c1), orc.back(p, c2), orc.remain(p, rest)]) / scale
                assert np.allclose(X[r, :3 * m], wf, rtol=1e-6)
                assert M[r, 0] == 1
                lb1, lb2 = b1[d, j], b2[d, j]
                if lb2 > lb1:
                    f, bk = orc.front(p, c1), orc.back(p, c2)
                    for q, (k, l) in enumerate(pairs):
                        g = p[:, k + 1:l].sum(axis=1)
                        order = [x for x in orc.johnson_lag_order(p[:, k], p[:, l], g) if x in rest]
                        if orc.pair_value(p, k, l, f, bk, order) == lb2:
                            hits[q] = 1
            if un:
                best = min(un, key=lambda j: (b2[d, j], j))
                tgt = [T[base + 1 + d * n + j, 0] for j in un]
                assert tgt == [1.0 if j == best else 0.0 for j in un]
        assert (T[base, 1:1 + len(pairs)] == hits).all(), (i, T[base, 1:1 + len(pairs)], hits)
        # a node without children has no pair targets: its mask stays zero
        assert (M[base, 1:1 + len(pairs)] == (1 if un else 0)).all() and M[base, 0] == 0
        for j in range(n):
            if j not in un:
                assert (X[base + 1 + j] == 0).all() and (M[base + 1 + j] == 0).all()


def test_traced_nodes_are_valid(pf):
    n, m = 12, 10
    p = inputs.make_instance(n, m, 17)
    inst = pf.pfsp_load_instance(p)
    perm, d1, d2, r = pf.pfsp_solve_trace(inst, 5000, stride=2, bound=pf.PFSP_LB2)
    assert 0 < len(d1) <= 5000
    assert len(d1) <= r["decomposed"] // 2 + r["explorers"] + 1
    for i in range(len(d1)):
        assert sorted(perm[i].tolist()) == list(range(n))
        assert d1[i] + d2[i] <= n - 1
    assert r["cmax"] == orc.bb_solve(p, bound=orc.LB2)["cmax"]


@pytest.mark.parametrize("n,m,seed", [(12, 10, 17), (11, 20, 3), (13, 5, 8)])
def test_learned_solver_is_exact(pf, n, m, seed):
    p = inputs.make_instance(n, m, seed)
    inst = pf.pfsp_load_instance(p)
    mlp = pf.pfsp_mlp_create(m, seed=seed)  # untrained: exactness must not depend on it
    opt = orc.bb_solve(p, bound=orc.LB2)["cmax"]
    capped = orc.bb_solve(p, bound=orc.LB2, init_ub=opt, capped=True)
    every = pf.PFSP_LEARN_CHILD_ORDER | pf.PFSP_LEARN_PAIR_ORDER | pf.PFSP_EARLY_EXIT | pf.PFSP_EARLY_EXIT_SLOTS
    r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt, branching=pf.PFSP_MINMIN_CAPPED, mlp=mlp,
                      learned=every)
    assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
    assert (r["decomposed"], r["bounded_children"]) == (capped["decomposed"], capped["bounded"])
    f = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, branching=pf.PFSP_MINMIN_CAPPED, mlp=mlp, learned=every)
    assert f["outcome"] == pf.PFSP_OPTIMAL and f["cmax"] == opt
    assert orc.makespan(p, f["perm"]) == opt
    g = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, mlp=mlp, learned=pf.PFSP_LEARN_CHILD_ORDER)
    assert g["cmax"] == opt


@pytest.mark.parametrize("n,m,seed", [(12, 10, 17), (11, 20, 3), (13, 5, 8), (12, 8, 6)])
def test_early_exit_keeps_the_tree(pf, n, m, seed):
    # a node one of whose directions is entirely at or above the incumbent
    # has no child below it under either MinMin rule, so stopping its LB2
    # sweep there changes no count, capped or not, whatever the pair order;
    # under MinBranch that direction has no survivor, so it is chosen unless
    # the other has none either, and then no child is explored either way
    p = inputs.make_instance(n, m, seed)
    inst = pf.pfsp_load_instance(p)
    opt = orc.bb_solve(p, bound=orc.LB2)["cmax"]
    rng = np.random.default_rng(seed)
    for order in (None, rng.permutation(m * (m - 1) // 2)):
        pf.pfsp_set_pair_order(inst, order)
        for rule in ("MINMIN", "MINMIN_CAPPED", "MINBRANCH"):
            want = orc.bb_solve(p, bound=orc.LB2, init_ub=opt, branching=getattr(orc, rule))
            for flags in (pf.PFSP_EARLY_EXIT, pf.PFSP_EARLY_EXIT | pf.PFSP_EARLY_EXIT_SLOTS):
                r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt, learned=flags,
                                  branching=getattr(pf, "PFSP_" + rule))
                assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
                got = (r["decomposed"], r["bounded_children"], r["pruned"])
                assert got == (want["decomposed"], want["bounded"], want["pruned"]), (order, rule, flags)
        f = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, learned=pf.PFSP_EARLY_EXIT)
        assert f["cmax"] == opt and orc.makespan(p, f["perm"]) == opt


@pytest.mark.parametrize("n,m,seed", [(12, 10, 17), (11, 20, 3), (13, 5, 8), (12, 8, 6), (33, 10, 4), (34, 5, 1)])
def test_early_exit_children_keeps_the_capped_tree(pf, n, m, seed):
    # PFSP_EARLY_EXIT_CHILDREN leaves out the jobs both of whose children
    # have an LB1 at or above the initial incumbent c; those children keep a
    # bound >= c, so min(bound, c) and the pruning are those of the full
    # sweep: capped MinMin builds the oracle's tree, whatever the pair order
    # (n = 34 runs the 64-bit-mask kernels, accumulators in shared memory)
    p = inputs.make_instance(n, m, seed)
    inst = pf.pfsp_load_instance(p)
    opt = orc.bb_solve(p, bound=orc.LB2)["cmax"]
    want = orc.bb_solve(p, bound=orc.LB2, init_ub=opt, branching=orc.MINMIN_CAPPED)
    base = pf.PFSP_EARLY_EXIT | pf.PFSP_EARLY_EXIT_CHILDREN
    rng = np.random.default_rng(seed)
    for order in (None, rng.permutation(m * (m - 1) // 2)):
        pf.pfsp_set_pair_order(inst, order)
        for flags in (base, base | pf.PFSP_EARLY_EXIT_SLOTS):
            r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt, learned=flags,
                              branching=pf.PFSP_MINMIN_CAPPED)
            assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
            got = (r["decomposed"], r["bounded_children"], r["pruned"])
            assert got == (want["decomposed"], want["bounded"], want["pruned"]), (order, flags)
        # under the other rules the tree may differ (tie-breaking sums), the
        # proof and the optimum may not
        for rule in (pf.PFSP_MINMIN, pf.PFSP_MINBRANCH):
            r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt, learned=base | pf.PFSP_EARLY_EXIT_SLOTS,
                              branching=rule)
            assert r["outcome"] == pf.PFSP_PROVEN_NO_BETTER
            f = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, learned=base | pf.PFSP_EARLY_EXIT_SLOTS, branching=rule)
            assert f["outcome"] == pf.PFSP_OPTIMAL and f["cmax"] == opt
            assert orc.makespan(p, f["perm"]) == opt
    pf.pfsp_set_pair_order(inst, None)


def test_early_exit_children_capped_proof_counts_20x10(pf):
    for g in json_golden():
        if g["proof_capped_decomposed"] > 300000:
            continue
        inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, g["seed"]))
        flags = pf.PFSP_EARLY_EXIT | pf.PFSP_EARLY_EXIT_CHILDREN | pf.PFSP_EARLY_EXIT_SLOTS
        r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"], learned=flags,
                          branching=pf.PFSP_MINMIN_CAPPED)
        assert r["decomposed"] == g["proof_capped_decomposed"], g["seed"]
        full = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"], branching=pf.PFSP_MINMIN_CAPPED)
        assert full["decomposed"] == r["decomposed"]
        assert r["lb2_slots"] <= full["lb2_slots"]


def test_early_exit_proof_counts_20x10(pf):
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "solve_20x10_lb2.json")))
    for g in gold["results"]:
        if g["proof_decomposed"] > 200000:
            continue
        inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, g["seed"]))
        r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"], learned=pf.PFSP_EARLY_EXIT)
        assert (r["decomposed"], r["bounded_children"], r["pruned"]) == (
            g["proof_decomposed"], g["proof_bounded"], g["proof_pruned"]), g["seed"]


def test_early_exit_skips_lb2_slots(pf):
    # the exit must actually fire: on a 20 x 10 proof (two 32-pair slots per
    # sweep) a large share of the nodes is decided by LB1 or the first slot
    g = [r for r in json_golden() if r["seed"] == 1][0]
    inst = pf.pfsp_load_instance(inputs.make_instance(20, 10, 1))
    full = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"])
    ee = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=g["optimum"], learned=pf.PFSP_EARLY_EXIT)
    assert full["decomposed"] == ee["decomposed"] == g["proof_decomposed"]
    assert full["lb2_slots"] == 2 * full["decomposed"]  # every node of this tree has children
    assert ee["lb2_slots"] < 0.8 * full["lb2_slots"], (ee["lb2_slots"], full["lb2_slots"])


def json_golden():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "solve_20x10_lb2.json")))["results"]


def test_pair_order_changes_no_bound(pf):
    n, m = 14, 10
    p = inputs.make_instance(n, m, 21)
    inst = pf.pfsp_load_instance(p)
    perm, d1, d2 = inputs.random_nodes(n, 3000, seed=4, dmax=6)
    a1, a2 = pf.pfsp_bound_batch(inst, 3, perm, d1, d2)
    mlp = pf.pfsp_mlp_create(m, seed=2)
    X0, T0, M0 = pf.pfsp_mlp_rows(inst, mlp, perm[:50], d1[:50], d2[:50])
    order = np.random.default_rng(1).permutation(m * (m - 1) // 2).astype(np.int32)
    pf.pfsp_set_pair_order(inst, order)
    assert (pf.pfsp_get_pair_order(inst) == order).all()
    b1, b2 = pf.pfsp_bound_batch(inst, 3, perm, d1, d2)
    assert (a1 == b1).all() and (a2 == b2).all()
    X1, T1, M1 = pf.pfsp_mlp_rows(inst, mlp, perm[:50], d1[:50], d2[:50])
    assert (X0 == X1).all() and (T0 == T1).all() and (M0 == M1).all()
    pf.pfsp_set_pair_order(inst, None)
    assert (pf.pfsp_get_pair_order(inst) == np.arange(m * (m - 1) // 2)).all()
    with pytest.raises(pf.PfspError):
        pf.pfsp_set_pair_order(inst, np.zeros(m * (m - 1) // 2, dtype=np.int32))


def test_learned_pair_order_ranks_network_scores(pf):
    n, m = 16, 10
    p = inputs.make_instance(n, m, 5)
    inst = pf.pfsp_load_instance(p)
    mlp = pf.pfsp_mlp_create(m, seed=9)
    perm, d1, d2, _ = pf.pfsp_solve_trace(inst, 400, stride=1, bound=pf.PFSP_LB2)
    score = pf.pfsp_mlp_pair_scores(inst, mlp, perm, d1, d2)
    # the same mean from the network's forward on the parent rows
    X, _, _ = pf.pfsp_mlp_rows(inst, mlp, perm, d1, d2)
    Y = pf.pfsp_mlp_forward(mlp, X[::1 + 2 * n])
    P = m * (m - 1) // 2
    want = (1.0 / (1.0 + np.exp(-Y[:, 1:1 + P].astype(np.float64)))).mean(axis=0)
    assert np.allclose(score, want, rtol=1e-5, atol=1e-6)
    order = pf.pfsp_learn_pair_order(inst, mlp, perm, d1, d2)
    assert sorted(order.tolist()) == list(range(P))
    assert (np.diff(score[order]) <= 0).all()
    assert (pf.pfsp_get_pair_order(inst) == order).all()


def test_learned_options_are_validated(pf):
    p = inputs.make_instance(8, 5, 1)
    inst = pf.pfsp_load_instance(p)
    with pytest.raises(pf.PfspError):  # slot checks without the early exit
        pf.pfsp_solve(inst, bound=2, learned=pf.PFSP_EARLY_EXIT_SLOTS)
    with pytest.raises(pf.PfspError):  # live-children sweep without the early exit
        pf.pfsp_solve(inst, bound=2, learned=pf.PFSP_EARLY_EXIT_CHILDREN)
    with pytest.raises(pf.PfspError):  # refused with MinSum
        pf.pfsp_solve(inst, bound=2, learned=pf.PFSP_EARLY_EXIT | pf.PFSP_EARLY_EXIT_CHILDREN,
                      branching=pf.PFSP_MINSUM)
    with pytest.raises(pf.PfspError):  # no network
        pf.pfsp_solve(inst, bound=2, learned=pf.PFSP_LEARN_CHILD_ORDER)
    other = pf.pfsp_mlp_create(10, seed=1)
    with pytest.raises(pf.PfspError):  # network for another m
        pf.pfsp_solve(inst, bound=2, mlp=other, learned=pf.PFSP_LEARN_PAIR_ORDER)


def test_training_on_solver_traces_beats_constant_predictor(pf):
    m = 10
    mlp = pf.pfsp_mlp_create(m, seed=5)
    Xs, Ts, Ms = [], [], []
    for seed in range(1, 5):
        inst = pf.pfsp_load_instance(inputs.make_instance(20, m, seed))
        perm, d1, d2, _ = pf.pfsp_solve_trace(inst, 1500, stride=3, bound=pf.PFSP_LB2)
        X, T, M = pf.pfsp_mlp_rows(inst, mlp, perm, d1, d2)
        keep = M.sum(axis=1) > 0
        Xs.append(X[keep]); Ts.append(T[keep]); Ms.append(M[keep])
    X, T, M = np.concatenate(Xs), np.concatenate(Ts), np.concatenate(Ms)
    rng = np.random.default_rng(0)
    idx = rng.permutation(len(X))
    cut = int(0.8 * len(X))
    tr, te = idx[:cut], idx[cut:]
    losses = pf.pfsp_mlp_train(mlp, X[tr], T[tr], M[tr], epochs=6, batch=2048, lr=2e-3, seed=2)
    assert losses[-1] < losses[0]
    # held-out masked BCE against the best constant per output column
    loss_net, _ = pf.pfsp_mlp_loss_grad(mlp, X[te], T[te], M[te])
    pr = (T[tr] * M[tr]).sum(0) / np.maximum(M[tr].sum(0), 1)
    pr = np.clip(pr, 1e-4, 1 - 1e-4)
    const = -(M[te] * (T[te] * np.log(pr) + (1 - T[te]) * np.log(1 - pr))).sum() / len(te)
    assert loss_net < const, (loss_net, const)


def test_learned_lb2_pair_subset_keeps_the_solve_exact(pf):
    # LB2 over the network's top pairs (scored on the root's children) is a
    # valid bound: the optimum is unchanged and the proof tree is the oracle's
    # for the same pairs
    n, m, P = 12, 10, 45
    p = inputs.make_instance(n, m, 17)
    inst = pf.pfsp_load_instance(p)
    mlp = pf.pfsp_mlp_create(m, seed=3)
    kept = pf.pfsp_learn_lb2_pairs(inst, mlp, keep=32)
    perm = np.array([[j] + [x for x in range(n) if x != j] if s == 0 else [x for x in range(n) if x != j] + [j]
                     for j in range(n) for s in (0, 1)], dtype=np.uint8)
    d1 = np.array([1 - s for j in range(n) for s in (0, 1)], dtype=np.uint8)
    d2 = 1 - d1
    score = pf.pfsp_mlp_pair_scores(inst, mlp, perm, d1, d2)
    assert list(kept) == list(np.argsort(-score, kind="stable")[:32])
    assert list(pf.pfsp_get_pair_order(inst)) == list(kept)
    opt = orc.bb_solve(p, bound=orc.LB2)["cmax"]
    want = orc.bb_solve(p, bound=orc.LB2, init_ub=opt, pairs=[int(q) for q in kept])
    r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt, learned=pf.PFSP_EARLY_EXIT)
    assert (r["decomposed"], r["bounded_children"], r["pruned"]) == (want["decomposed"], want["bounded"],
                                                                      want["pruned"])
    assert r["lb2_slots"] <= r["decomposed"]
    # the subset in the plain kernel: one 32-pair slot per decomposition
    r0 = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt)
    assert (r0["decomposed"], r0["bounded_children"], r0["pruned"]) == (want["decomposed"], want["bounded"],
                                                                         want["pruned"])
    assert r0["lb2_slots"] == r0["decomposed"]
    f = pf.pfsp_solve(inst, bound=pf.PFSP_LB2)
    assert f["cmax"] == opt and orc.makespan(p, f["perm"]) == opt
    assert len(pf.pfsp_learn_lb2_pairs(inst, mlp, keep=100)) == P  # keep >= P: every pair


def test_learned_solver_workflow_keeps_the_capped_tree(pf):
    # the learned solver of the comparison: the network orders the pairs
    # (scores on the root's children), the sweep exits early per child; under
    # capped MinMin its tree is the oracle's, under MinMin the optimum is
    from paper_2012_09511_gb300 import learned
    n, m = 13, 10
    p = inputs.make_instance(n, m, 45)
    inst = pf.pfsp_load_instance(p)
    mlp = pf.pfsp_mlp_create(m, seed=4)
    order = learned.order_pairs(pf, inst, mlp)
    assert sorted(order.tolist()) == list(range(m * (m - 1) // 2))
    assert (pf.pfsp_get_pair_order(inst) == order).all()
    perm, d1, d2 = learned.root_children(n)
    score = pf.pfsp_mlp_pair_scores(inst, mlp, perm, d1, d2)
    assert (np.diff(score[order]) <= 0).all()
    opt = orc.bb_solve(p, bound=orc.LB2)["cmax"]
    want = orc.bb_solve(p, bound=orc.LB2, init_ub=opt, branching=orc.MINMIN_CAPPED)
    for slots in (False, True):
        r = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, init_ub=opt, branching=pf.PFSP_MINMIN_CAPPED,
                          **learned.learned_options(pf, slot_checks=slots))
        assert (r["decomposed"], r["bounded_children"], r["pruned"]) == (want["decomposed"], want["bounded"],
                                                                         want["pruned"])
        f = pf.pfsp_solve(inst, bound=pf.PFSP_LB2, **learned.learned_options(pf, slot_checks=slots))
        assert f["cmax"] == opt and orc.makespan(p, f["perm"]) == opt
