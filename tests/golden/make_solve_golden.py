"""Write tests/golden/solve_20x10_lb2.json: oracle results for the exact-solve
workload (n = 20 jobs, m = 10 machines, times uniform in [1, 99], seeds 1..10,
LB2 with MinMin).

For every seed the oracle first solves from its NEH schedule (optimum and
optimal permutation), then re-runs in proof mode with the incumbent set to the
optimum, which fixes the explored tree: its decomposed and bounded counts are
the values the device solver must reproduce exactly.  Only oracle/ is called.
Run from the repository root:  python tests/golden/make_solve_golden.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N, M, SEEDS = 20, 10, range(1, 11)


def one(seed):
    import oracle as orc
    from paper_2012_09511_gb300 import inputs
    p = inputs.make_instance(N, M, seed)
    t = time.time()
    r = orc.bb_solve(p, bound=orc.LB2)
    t1 = time.time() - t
    assert r["outcome"] == orc.OPTIMAL
    t = time.time()
    q = orc.bb_solve(p, bound=orc.LB2, init_ub=r["cmax"])
    t2 = time.time() - t
    qc = orc.bb_solve(p, bound=orc.LB2, init_ub=r["cmax"], capped=True)
    assert q["outcome"] == orc.PROVEN_NO_BETTER
    return {"seed": seed, "optimum": r["cmax"], "perm": [int(x) for x in r["perm"]],
            "proof_decomposed": q["decomposed"], "proof_bounded": q["bounded"], "proof_leaves": q["leaves"],
            "proof_pruned": q["pruned"], "proof_capped_decomposed": qc["decomposed"],
            "oracle_find_seconds": round(t1, 2), "oracle_proof_seconds": round(t2, 2)}


def main():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(SEEDS), os.cpu_count() or 1)) as pool:
        res = pool.map(one, list(SEEDS))
    out = {"workload": "n=20, m=10, uniform [1,99], seeds 1..10, LB2 + MinMin (uncapped and capped)",
           "generator": "paper_2012_09511_gb300.inputs.make_instance(20, 10, seed)",
           "script": "tests/golden/make_solve_golden.py", "results": res}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "solve_20x10_lb2.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
