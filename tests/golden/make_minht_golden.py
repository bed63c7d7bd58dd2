"""Write tests/golden/solve_lb1_minht.json: oracle proof-mode trees of a few
LB1 instances with and without the heads and tails refinement of LB1 (the
option of pfsp_options.lb1_minht; not in the paper).

Each instance is solved by the oracle from NEH (optimum), then in proof mode
at the optimum with the plain LB1 and with the refined one.  Only oracle/ is
called.  Run from the repository root:  python tests/golden/make_minht_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CASES = [(12, 6, 20), (12, 6, 21), (13, 6, 21), (14, 8, 21), (12, 10, 21), (12, 10, 22), (15, 8, 30)]


def main():
    import oracle as orc
    from paper_2012_09511_gb300 import inputs
    orc.build()
    res = []
    for n, m, seed in CASES:
        p = inputs.make_instance(n, m, seed)
        opt = orc.bb_solve(p, bound=orc.LB1)["cmax"]
        out = {"n": n, "m": m, "seed": seed, "optimum": opt}
        for name, minht in (("plain", False), ("minht", True)):
            t = time.time()
            q = orc.bb_solve(p, bound=orc.LB1, init_ub=opt, minht=minht)
            assert q["outcome"] == orc.PROVEN_NO_BETTER
            out[name] = {"decomposed": q["decomposed"], "bounded": q["bounded"],
                         "oracle_proof_seconds": round(time.time() - t, 2)}
        res.append(out)
    doc = {"workload": "LB1 proofs at the optimum, plain and with the heads and tails refinement",
           "generator": "paper_2012_09511_gb300.inputs.make_instance(n, m, seed)",
           "script": "tests/golden/make_minht_golden.py", "results": res}
    with open(os.path.join(HERE, "solve_lb1_minht.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
