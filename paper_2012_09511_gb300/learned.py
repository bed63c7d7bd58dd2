"""Learned ordering workflow: traces -> training rows -> network -> solves.

Orchestration only; every step runs in the library's kernels:
pfsp_solve_trace records nodes the solver decomposes, pfsp_mlp_rows builds
the training rows on the GPU, pfsp_mlp_train trains the network on the GPU,
pfsp_learn_lb2_pairs scores the machine pairs with the network, and
pfsp_solve runs the plain and the learned solvers.

The learned solver restricts LB2 to the machine pairs that the network
predicts most often give a child's LB2 (scored on the root's children; half
of the 32-pair slots: one of two at m = 10, three of six at m = 20).  A
subset LB2 is still a lower bound, so the search stays exact and its optimum
is always the plain solver's; the comparison reports the time to the proven
optimum (wall time, ranking included) and the decomposed-node counts of both.
The early exit of the LB2 sweep (a node one of whose directions has every
child at or above the incumbent needs no sweep) and the network's row order
are reported as ablations.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs

LEARNED_ALL = 1 | 2 | 4  # child order | pair order | early exit


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


def _run(pfsp, inst, **kw):
    t = time.perf_counter()
    r = pfsp.pfsp_solve(inst, **kw)
    return r, time.perf_counter() - t


def learned_pairs(pfsp, inst, mlp, keep=None):
    """LB2 of `inst` restricted to the `keep` machine pairs the network scores
    highest on the root's children (pfsp_learn_lb2_pairs).  By default half of
    the 32-pair slots, rounded up, are kept: 32 of 45 pairs at m = 10 (one slot
    of two), 96 of 190 at m = 20 (three of six); measured on proofs, fewer
    pairs weaken the bound more than they save.  Nothing changes when the
    instance has at most `keep` pairs.  Returns the pairs kept, or None."""
    P = inst.m * (inst.m - 1) // 2
    if keep is None:
        keep = 32 * (((P + 31) // 32 + 1) // 2)
    if P <= keep:
        pfsp.pfsp_set_lb2_pairs(inst, None)
        return None
    return pfsp.pfsp_learn_lb2_pairs(inst, mlp, keep=keep)


def learned_options(pfsp):
    """pfsp_solve options of the learned solver (the LB2 pair subset is set on
    the instance by learned_pairs): none beyond the subset.  The early exit of
    the sweep runs in a kernel of its own whose checks cost instruction fetch;
    with the subset it is 1.0x at m = 10 and 0.9x at m = 20, so it stays an
    ablation."""
    return {}


def solve_variants(pfsp, p, mlp, time_limit_s=30.0, depths=None, init_ub=None):
    """Plain and learned solves of one instance (LB2), from its NEH schedule or,
    with init_ub, in proof mode.

    plain: the full-pair LB2 solver, pairs in index order.
    learned: LB2 over the network's top pairs (learned_pairs: half of the
    32-pair slots); its wall time includes the ranking.
    Ablations: early exit alone, and in finding mode the network's row order
    at each depth of `depths` (with early exit, all pairs)."""
    n = p.shape[0]
    depths = depths or [max(1, n // 4)]
    inst = pfsp.pfsp_load_instance(p)
    base = dict(bound=2, time_limit_s=time_limit_s)
    if init_ub is not None:
        base["init_ub"] = int(init_ub)
    out = {}

    def record(name, r, wall, extra_wall=0.0):
        out[name] = {"cmax": r["cmax"], "outcome": r["outcome"], "seconds": r["kernel_seconds"],
                     "wall_seconds": wall + extra_wall, "decomposed": r["decomposed"],
                     "bounded": r["bounded_children"], "lb2_slots": r["lb2_slots"]}

    pfsp.pfsp_set_lb2_pairs(inst, None)
    record("plain", *_run(pfsp, inst, **base))
    record("early_exit", *_run(pfsp, inst, learned=pfsp.PFSP_EARLY_EXIT, **base))
    if init_ub is None:
        for d in depths:
            record("child_order_depth_%d" % d,
                   *_run(pfsp, inst, learned=pfsp.PFSP_EARLY_EXIT | pfsp.PFSP_LEARN_CHILD_ORDER, mlp=mlp,
                         learn_depth=d, **base))
    t = time.perf_counter()
    kept = learned_pairs(pfsp, inst, mlp)
    t_rank = time.perf_counter() - t
    record("learned", *_run(pfsp, inst, **learned_options(pfsp), **base), extra_wall=t_rank)
    out["ranking_wall_seconds"] = t_rank
    out["pairs_kept"] = None if kept is None else [int(q) for q in kept]
    pfsp.pfsp_set_lb2_pairs(inst, None)
    return out


def compare(pfsp, shapes=((50, 5), (30, 10)), seeds=range(1, 6), train_seeds=range(1, 11), time_limit_s=30.0,
            depth_fracs=(4,), proof=False, mlps=None):
    """Time to the proven optimum, plain vs learned, on the given shapes.

    The m-machine network is trained on traces of 20-job instances with the same
    m (seeds train_seeds), unless mlps maps m to a trained network; the
    evaluation instances are n x m with seeds 100 + s, disjoint from training.
    proof=False solves from NEH (find and prove); proof=True first finds the
    optimum with the plain solver, then times both solvers proving it (incumbent
    at the optimum, a fixed tree)."""
    report = {}
    for n, m in shapes:
        if mlps and m in mlps:
            mlp, info = mlps[m], {"reused": True}
        else:
            t = time.perf_counter()
            train = [inputs.make_instance(20, m, s) for s in train_seeds]
            mlp, info = train_network(pfsp, m, train)
            info["seconds"] = time.perf_counter() - t
        rows = []
        for s in seeds:
            p = inputs.make_instance(n, m, 100 + s)
            ub = None
            if proof:
                inst = pfsp.pfsp_load_instance(p)
                f = pfsp.pfsp_solve(inst, bound=2, time_limit_s=time_limit_s)
                if f["outcome"] != pfsp.PFSP_OPTIMAL:
                    continue
                ub = f["cmax"]
            r = solve_variants(pfsp, p, mlp, time_limit_s=time_limit_s,
                               depths=[max(1, n // f) for f in depth_fracs], init_ub=ub)
            r["seed"] = 100 + s
            r["same_optimum"] = len({v["cmax"] for v in r.values() if isinstance(v, dict)}) == 1
            rows.append(r)
        want = pfsp.PFSP_PROVEN_NO_BETTER if proof else pfsp.PFSP_OPTIMAL
        done = [r for r in rows if all(r[k]["outcome"] == want for k in ("plain", "learned"))]

        def tot(key, field):
            return sum(r[key][field] for r in done)

        t_plain, t_learn = tot("plain", "wall_seconds"), tot("learned", "wall_seconds")
        t_rank = sum(r["ranking_wall_seconds"] for r in done)
        k_plain, k_learn = tot("plain", "seconds"), tot("learned", "seconds")
        n_plain, n_learn = tot("plain", "decomposed"), tot("learned", "decomposed")
        report["%dx%d" % (n, m)] = {
            "mode": "proof" if proof else "find", "training": info, "instances": rows,
            "solved_by_both": len(done),
            "wall_plain_s": t_plain, "wall_learned_s": t_learn,
            "speedup_wall": (t_plain / t_learn) if t_learn > 0 else None,
            # the network's share of the learned solver's time: it runs once per
            # instance, on the root's children, to rank the machine pairs
            "ranking_wall_s": t_rank,
            "mlp_share_of_learned_wall": (t_rank / t_learn) if t_learn > 0 else None,
            "kernel_plain_s": k_plain, "kernel_learned_s": k_learn,
            "speedup_kernel": (k_plain / k_learn) if k_learn > 0 else None,
            "node_ratio_learned_over_plain": (n_learn / n_plain) if n_plain > 0 else None,
            "ablation_wall_s": {key: tot(key, "wall_seconds") for key in done[0] if isinstance(done[0][key], dict)}
            if done else {},
        }
    return report
