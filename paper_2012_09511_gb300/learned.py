"""Learned ordering workflow: traces -> training rows -> network -> solves.

Orchestration only; every step runs in the library's kernels:
pfsp_solve_trace records nodes the solver decomposes, pfsp_mlp_rows builds
the training rows on the GPU, pfsp_mlp_train trains the network on the GPU,
pfsp_learn_pair_order ranks the machine pairs with the network, and
pfsp_solve runs the plain and the learned solvers.

The learned solver (not in the paper) orders the LB2 sweep and exits it early:
  * order: the network scores every machine pair on the root's 2n children
    (its mean probability that the pair gives a child's LB2) and the instance's
    pairs are swept best first (pfsp_learn_pair_order);
  * early exit: a node one of whose directions has every child at or above
    the incumbent needs no sweep (reading R14); otherwise only the jobs with a
    child still below it are evaluated (PFSP_EARLY_EXIT_CHILDREN), and, with
    slot checks (on by default from four 32-pair slots, m >= 15), a job whose
    two children are decided leaves the later slots and the sweep stops after
    the slot at which one direction is decided: there the network's order
    acts.
Every child that can survive gets its exact full-pair LB2, so pruning stays
exact and the plain full-pair LB2 solver is the reference: under capped MinMin the
two build the same tree (node counts equal, checked), under the paper's
MinMin the tie-breaking sums of decided children may differ and the node
inflation is reported.  The comparison proves a known optimum (incumbent at
the optimum, a fixed tree) and reports the median of repeated solves.
Ablations: the same early exit with the pairs in index order (what the
network's order adds) and LB2 restricted to the network's top pairs (a weaker
bound, the learned pair subset).
"""
from __future__ import annotations

import statistics
import time

import numpy as np

from . import inputs

LEARNED_ALL = 1 | 2 | 4  # child order | pair order | early exit
EARLY_EXIT, EARLY_EXIT_SLOTS, EARLY_EXIT_CHILDREN = 4, 8, 16

# The 30 x 10 instances of the comparison: seeds 101 upwards, the first ten
# whose proof of the optimum takes the plain solver at least 50 ms of kernel
# time on one GB300 (most 30 x 10 proofs take a few milliseconds).
SEEDS_30X10 = (135, 232, 370, 415, 421, 457, 564, 583, 642, 672)


def collect_rows(pfsp, instances, mlp, nodes_per_instance=4000, stride=2, bound=2, time_limit_s=5.0):
    """Training rows from traces of the solver on `instances` (p matrices)."""
    Xs, Ts, Ms = [], [], []
    for p in instances:
        inst = pfsp.pfsp_load_instance(p)
        perm, d1, d2, _ = pfsp.pfsp_solve_trace(inst, nodes_per_instance, stride=stride, bound=bound,
                                                time_limit_s=time_limit_s)
        if len(d1) == 0:
            continue
        X, T, M = pfsp.pfsp_mlp_rows(inst, mlp, perm, d1, d2)
        keep = M.sum(axis=1) > 0
        Xs.append(X[keep])
        Ts.append(T[keep])
        Ms.append(M[keep])
    return np.concatenate(Xs), np.concatenate(Ts), np.concatenate(Ms)


def train_network(pfsp, m, train_instances, seed=0, epochs=8, batch=4096, lr=2e-3, **trace_kw):
    """A network for m machines trained on the solver's traces of train_instances."""
    mlp = pfsp.pfsp_mlp_create(m, seed=seed)
    X, T, M = collect_rows(pfsp, train_instances, mlp, **trace_kw)
    losses = pfsp.pfsp_mlp_train(mlp, X, T, M, epochs=epochs, batch=batch, lr=lr, seed=seed + 1)
    return mlp, {"rows": int(len(X)), "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1])}


def root_children(n):
    """The root's 2n children in the layout of pfsp_bound_batch: job j first
    (forward, d1 = 1) and job j last (backward, d2 = 1)."""
    perm = np.empty((2 * n, n), dtype=np.uint8)
    d1 = np.zeros(2 * n, dtype=np.uint8)
    d2 = np.zeros(2 * n, dtype=np.uint8)
    for j in range(n):
        rest = [q for q in range(n) if q != j]
        perm[j] = [j] + rest
        d1[j] = 1
        perm[n + j] = rest + [j]
        d2[n + j] = 1
    return perm, d1, d2


def order_pairs(pfsp, inst, mlp):
    """Sweep the instance's pairs in the network's order (mean pair probability
    over the root's children, best first); returns the order, or None when
    every pair fits one 32-pair slot (m <= 8): the sweep then evaluates all of
    them at once and no order can change its work, so the network is not run."""
    if inst.m * (inst.m - 1) // 2 <= 32:
        pfsp.pfsp_set_pair_order(inst, None)
        return None
    perm, d1, d2 = root_children(inst.n)
    return pfsp.pfsp_learn_pair_order(inst, mlp, perm, d1, d2)


def slot_checks_for(m):
    """Whether the learned solver checks after every 32-pair slot for m
    machines: from four slots on (m >= 15).  Measured on one GB300: at m = 20
    the checks with the network's pair order are the fastest variant (18 x 20
    proofs 1.8 % below the same early exit without them); at m = 10 (two slots,
    the second holding 13 pairs) they cost about what they save."""
    return m * (m - 1) // 2 > 96


def learned_options(pfsp, slot_checks=None, m=None):
    """pfsp_solve options of the learned solver (the pair order is set on the
    instance by order_pairs): the early exit per child, and the check after
    every 32-pair slot when slot_checks says so (None: slot_checks_for(m))."""
    flags = pfsp.PFSP_EARLY_EXIT | pfsp.PFSP_EARLY_EXIT_CHILDREN
    if slot_checks is None:
        slot_checks = m is not None and slot_checks_for(m)
    if slot_checks:
        flags |= pfsp.PFSP_EARLY_EXIT_SLOTS
    return {"learned": flags}


def learned_pairs(pfsp, inst, mlp, keep=None):
    """LB2 of `inst` restricted to the `keep` machine pairs the network scores
    highest on the root's children (pfsp_learn_lb2_pairs; the learned pair
    subset, a weaker bound).  By default half of the 32-pair slots, rounded up.
    Nothing changes when the instance has at most `keep` pairs.  Returns the
    pairs kept, or None."""
    P = inst.m * (inst.m - 1) // 2
    if keep is None:
        keep = 32 * (((P + 31) // 32 + 1) // 2)
    if P <= keep:
        pfsp.pfsp_set_lb2_pairs(inst, None)
        return None
    return pfsp.pfsp_learn_lb2_pairs(inst, mlp, keep=keep)


def _median_solve(pfsp, inst, reps, **kw):
    """Median kernel and wall seconds of `reps` solves (after one untimed)."""
    pfsp.pfsp_solve(inst, **kw)
    ks, ws, r = [], [], None
    for _ in range(reps):
        t = time.perf_counter()
        r = pfsp.pfsp_solve(inst, **kw)
        ws.append(time.perf_counter() - t)
        ks.append(r["kernel_seconds"])
    return r, statistics.median(ks), statistics.median(ws)


def proof_variants(pfsp, p, opt, mlp, rule, reps=3, slot_checks=None, subset=True):
    """Proofs of the optimum `opt` of instance p (LB2, branching `rule`) by the
    plain full-pair solver, the learned solver and the ablations (slot checks:
    see learned_options)."""
    inst = pfsp.pfsp_load_instance(p)
    ee = learned_options(pfsp, slot_checks, m=inst.m)
    base = dict(bound=2, init_ub=int(opt), branching=rule)
    out = {}

    def record(name, r, k, w, extra_wall=0.0):
        assert r["outcome"] == pfsp.PFSP_PROVEN_NO_BETTER, (name, r["outcome"])
        out[name] = {"kernel_s": k, "wall_s": w + extra_wall, "decomposed": int(r["decomposed"]),
                     "lb2_slots": int(r["lb2_slots"])}

    pfsp.pfsp_set_lb2_pairs(inst, None)
    record("plain", *_median_solve(pfsp, inst, reps, **base))
    record("early_exit_index_order", *_median_solve(pfsp, inst, reps, **ee, **base))
    t = time.perf_counter()
    order_pairs(pfsp, inst, mlp)
    t_rank = time.perf_counter() - t
    record("learned", *_median_solve(pfsp, inst, reps, **ee, **base),
           extra_wall=t_rank)
    out["ranking_wall_s"] = t_rank
    if subset:
        pfsp.pfsp_set_pair_order(inst, None)
        t = time.perf_counter()
        kept = learned_pairs(pfsp, inst, mlp)
        t_sub = time.perf_counter() - t
        if kept is not None:
            record("pair_subset", *_median_solve(pfsp, inst, reps, **base), extra_wall=t_sub)
        pfsp.pfsp_set_lb2_pairs(inst, None)
    return out


def compare_proofs(pfsp, cases, mlps, rules=(("minmin", 0),), reps=3, slot_checks=None, subset_rules=("minmin",)):
    """Time-to-proof of the plain full-pair LB2 solver and of the learned solver.

    cases: {name: (n, m, seeds)}; the optimum of each instance is found first
    by the plain solver from NEH, then each variant proves it `reps` times
    (median).  rules: (name, PFSP branching rule) pairs."""
    report = {}
    for name, (n, m, seeds) in cases.items():
        rows = []
        for s in seeds:
            p = inputs.make_instance(n, m, s)
            f = pfsp.pfsp_solve(pfsp.pfsp_load_instance(p), bound=2, time_limit_s=30.0)
            if f["outcome"] != pfsp.PFSP_OPTIMAL:
                continue
            row = {"seed": s, "optimum": int(f["cmax"])}
            for rname, rule in rules:
                row[rname] = proof_variants(pfsp, p, f["cmax"], mlps[m], rule, reps=reps, slot_checks=slot_checks,
                                            subset=rname in subset_rules)
            rows.append(row)
        rep = {"instances": len(rows), "seeds": [r["seed"] for r in rows]}
        for rname, _ in rules:
            keys = [k for k, v in rows[0][rname].items() if isinstance(v, dict)] if rows else []
            tot = {k: sum(r[rname][k]["kernel_s"] for r in rows) for k in keys}
            wall = {k: sum(r[rname][k]["wall_s"] for r in rows) for k in keys}
            nodes = {k: sum(r[rname][k]["decomposed"] for r in rows) for k in keys}
            per = [r[rname]["plain"]["kernel_s"] / r[rname]["learned"]["kernel_s"] for r in rows]
            rep[rname] = {
                "kernel_s": tot, "wall_s": wall, "decomposed": nodes,
                "speedup_kernel": tot["plain"] / tot["learned"] if rows else None,
                "speedup_wall": wall["plain"] / wall["learned"] if rows else None,
                "speedup_kernel_per_seed_median": statistics.median(per) if per else None,
                "seeds_faster": int(sum(x > 1.0 for x in per)),
                "node_ratio_learned_over_plain": nodes["learned"] / nodes["plain"] if rows else None,
                "ranking_wall_s": sum(r[rname]["ranking_wall_s"] for r in rows),
            }
        report[name] = rep
    return report


def compare_finding(pfsp, n, m, seeds, mlp, rule=0):
    """Time to the proven optimum from the NEH schedule (finding mode), plain
    full-pair LB2 against the learned solver, one solve each per instance
    (finding-mode trees depend on when each explorer meets the incumbents, so
    they vary from run to run); optima must agree."""
    tot = {"plain": 0.0, "learned": 0.0}
    nodes = {"plain": 0, "learned": 0}
    same = True
    for s in seeds:
        inst = pfsp.pfsp_load_instance(inputs.make_instance(n, m, s))
        pfsp.pfsp_set_pair_order(inst, None)
        a = pfsp.pfsp_solve(inst, bound=2, branching=rule, time_limit_s=30.0)
        order_pairs(pfsp, inst, mlp)
        b = pfsp.pfsp_solve(inst, bound=2, branching=rule, time_limit_s=30.0, **learned_options(pfsp, m=m))
        same &= a["cmax"] == b["cmax"] and a["outcome"] == b["outcome"] == pfsp.PFSP_OPTIMAL
        for k, r in (("plain", a), ("learned", b)):
            tot[k] += r["kernel_seconds"]
            nodes[k] += int(r["decomposed"])
    return {"kernel_s": tot, "decomposed": nodes, "same_optima": bool(same),
            "speedup_kernel": tot["plain"] / tot["learned"] if tot["learned"] > 0 else None}
