"""Learned ordering workflow: traces -> training rows -> network -> solves.

Orchestration only; every step runs in the library's kernels:
pfsp_solve_trace records nodes the solver decomposes, pfsp_mlp_rows builds
the training rows on the GPU, pfsp_mlp_train trains the network on the GPU,
and pfsp_solve runs the plain and the learned solvers.

The learned solver uses the capped MinMin rule, sweeps LB2's 32-pair slots in
the order of the network's pair logits and stops the sweep once every child's
bound reaches the cap, and orders each new row by the network's descend-first
logits.  Its optimum is always the plain solver's; the comparison reports the
time to the proven optimum and the decomposed-node counts of both.
"""
from __future__ import annotations

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


def solve_variants(pfsp, p, mlp, time_limit_s=30.0, depths=None):
    """Plain and learned solves of one instance from its NEH schedule (LB2).

    `learned` uses every learned option with the network ordering the rows of
    the first `depth` levels (depth = depths[0], default n / 3); the other
    entries are ablations: the capped rule and early exit without the network,
    and the network's row order alone at each depth of `depths`."""
    n = p.shape[0]
    depths = depths or [max(1, n // 3)]
    inst = pfsp.pfsp_load_instance(p)
    runs = {
        "plain": dict(),
        "capped_static_early_exit": dict(branching=1, learned=4),
        "learned": dict(branching=1, learned=LEARNED_ALL, mlp=mlp, learn_depth=depths[0]),
    }
    for d in depths:
        runs["child_order_depth_%d" % d] = dict(learned=1, mlp=mlp, learn_depth=d)
    out = {}
    for name, kw in runs.items():
        r = pfsp.pfsp_solve(inst, bound=2, time_limit_s=time_limit_s, **kw)
        out[name] = {"cmax": r["cmax"], "outcome": r["outcome"], "seconds": r["kernel_seconds"],
                     "decomposed": r["decomposed"], "bounded": r["bounded_children"]}
    return out


def compare(pfsp, shapes=((50, 5), (30, 10)), seeds=range(1, 6), train_seeds=range(1, 11), time_limit_s=30.0,
            depth_fracs=(3,)):
    """Time to the proven optimum, plain vs learned, on the given shapes.

    The m-machine network is trained on traces of 20-job instances with the same
    m (seeds train_seeds); the evaluation instances are n x m with seeds
    100 + s, disjoint from training."""
    report = {}
    for n, m in shapes:
        train = [inputs.make_instance(20, m, s) for s in train_seeds]
        mlp, info = train_network(pfsp, m, train)
        rows = []
        for s in seeds:
            p = inputs.make_instance(n, m, 100 + s)
            r = solve_variants(pfsp, p, mlp, time_limit_s=time_limit_s,
                               depths=[max(1, n // f) for f in depth_fracs])
            r["seed"] = 100 + s
            r["same_optimum"] = len({v["cmax"] for v in r.values() if isinstance(v, dict)}) == 1
            rows.append(r)
        done = [r for r in rows if all(r[k]["outcome"] == 0 for k in ("plain", "learned"))]
        t_plain = sum(r["plain"]["seconds"] for r in done)
        t_learn = sum(r["learned"]["seconds"] for r in done)
        n_plain = sum(r["plain"]["decomposed"] for r in done)
        n_learn = sum(r["learned"]["decomposed"] for r in done)
        report["%dx%d" % (n, m)] = {
            "training": info, "instances": rows, "solved_by_both": len(done),
            "time_plain_s": t_plain, "time_learned_s": t_learn,
            "speedup": (t_plain / t_learn) if t_learn > 0 else None,
            "node_ratio_learned_over_plain": (n_learn / n_plain) if n_plain > 0 else None,
        }
    return report
