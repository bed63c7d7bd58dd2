"""Write tests/golden/batch256_lb2.json: oracle optima of the uneven batch.

Instance i (i = 0..255) has the shape inputs.batch_instance_shape(i) (n in
12..20, m in {5, 10, 20}) and processing times inputs.make_instance(n, m,
1000 + i).  The oracle solves each from its NEH schedule with LB2 and MinMin;
an instance that needs more than NODE_LIMIT decompositions is then proved in a
second oracle pass: the incumbent the first pass reached (a complete schedule
whose makespan the oracle recomputes) becomes the exclusive initial upper bound
of a fresh search with PROOF_LIMIT decompositions.  That search explores a
subset of the first one's tree and ends either with nothing below the incumbent
(the incumbent is optimal) or with a better schedule and a completed search.
An instance that neither pass finishes is recorded as unverified (no optimum),
never guessed.  Only oracle/ is called.  The script resumes from a partial file,
so it can be re-run until every instance is done:
    python tests/golden/make_batch_golden.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch256_lb2.json")
COUNT, NODE_LIMIT, PROOF_LIMIT = 256, 3_000_000, 400_000_000


def one(i):
    import oracle as orc
    from paper_2012_09511_gb300 import inputs
    n, m = inputs.batch_instance_shape(i)
    p = inputs.make_instance(n, m, 1000 + i)
    t = time.time()
    r = orc.bb_solve(p, bound=orc.LB2, node_limit=NODE_LIMIT)
    rec = {"i": i, "n": n, "m": m, "decomposed": r["decomposed"], "oracle_seconds": round(time.time() - t, 2)}
    if r["outcome"] == orc.OPTIMAL:
        rec["optimum"] = r["cmax"]
        return rec
    assert orc.makespan(p, r["perm"]) == r["cmax"]
    t = time.time()
    q = orc.bb_solve(p, bound=orc.LB2, init_ub=r["cmax"], node_limit=PROOF_LIMIT)
    rec.update(incumbent=r["cmax"], proof_decomposed=q["decomposed"],
               proof_seconds=round(time.time() - t, 2))
    if q["outcome"] == orc.PROVEN_NO_BETTER:
        rec["optimum"] = r["cmax"]
    elif q["outcome"] == orc.OPTIMAL:
        assert orc.makespan(p, q["perm"]) == q["cmax"] < r["cmax"]
        rec["optimum"] = q["cmax"]
    else:
        rec["unverified"] = "oracle stopped at %d + %d decompositions" % (NODE_LIMIT, PROOF_LIMIT)
    return rec


def main():
    import oracle
    oracle.build()
    done = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            done = {r["i"]: r for r in json.load(f)["results"]}
    todo = [i for i in range(COUNT) if i not in done or
            ("unverified" in done[i] and done[i].get("proof_decomposed", 0) < PROOF_LIMIT)]
    todo.sort(key=lambda i: -done[i]["decomposed"] if i in done else 0)
    ctx = mp.get_context("spawn")
    workers = int(os.environ.get("GOLDEN_WORKERS", max(1, (os.cpu_count() or 2) - 1)))
    with ctx.Pool(workers) as pool:
        for rec in pool.imap_unordered(one, todo):
            done[rec["i"]] = rec
            with open(OUT + ".tmp", "w") as f:
                json.dump({"workload": "256 instances, shape batch_instance_shape(i), times make_instance(n, m, 1000+i), "
                                       "LB2 + MinMin from NEH", "script": "tests/golden/make_batch_golden.py",
                           "node_limit": NODE_LIMIT, "proof_limit": PROOF_LIMIT, "results": [done[k] for k in sorted(done)]}, f, indent=0)
            os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()
