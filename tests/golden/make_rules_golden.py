"""Write tests/golden/solve_20x10_rules.json: oracle proof-mode trees of the
exact-solve workload (n = 20 jobs, m = 10 machines, times uniform in [1, 99],
seeds 1..10, LB2) under the MinBranch and MinSum branching rules (readings of
the rules Table 4 names; MinMin's are in solve_20x10_lb2.json).

For every seed the incumbent is fixed at the optimum recorded in
solve_20x10_lb2.json, which fixes each rule's tree: its decomposed and bounded
counts are the values the device solver must reproduce.  Only oracle/ is
called.  Run from the repository root:  python tests/golden/make_rules_golden.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, M, SEEDS = 20, 10, range(1, 11)


def one(job):
    seed, opt = job
    import oracle as orc
    from paper_2012_09511_gb300 import inputs
    p = inputs.make_instance(N, M, seed)
    out = {"seed": seed, "optimum": opt}
    for name, rule in (("minbranch", orc.MINBRANCH), ("minsum", orc.MINSUM)):
        t = time.time()
        q = orc.bb_solve(p, bound=orc.LB2, init_ub=opt, branching=rule)
        assert q["outcome"] == orc.PROVEN_NO_BETTER
        out[name] = {"decomposed": q["decomposed"], "bounded": q["bounded"], "pruned": q["pruned"],
                     "oracle_proof_seconds": round(time.time() - t, 2)}
    return out


def main():
    import oracle
    oracle.build()
    with open(os.path.join(HERE, "solve_20x10_lb2.json")) as f:
        opt = {r["seed"]: r["optimum"] for r in json.load(f)["results"]}
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(SEEDS), os.cpu_count() or 1)) as pool:
        res = pool.map(one, [(s, opt[s]) for s in SEEDS])
    out = {"workload": "n=20, m=10, uniform [1,99], seeds 1..10, LB2, proof mode at the optimum, "
                       "MinBranch and MinSum",
           "generator": "paper_2012_09511_gb300.inputs.make_instance(20, 10, seed)",
           "script": "tests/golden/make_rules_golden.py", "results": res}
    with open(os.path.join(HERE, "solve_20x10_rules.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
