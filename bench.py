"""Benchmark of the PFSP branch-and-bound hot path on GB300.

Workload (one step): the 20 x 20 bounding batch -- n = 20 jobs, m = 20
machines, processing times uniform in [1, 99], 4,194,304 random partial
schedules with prefix and suffix depths uniform in {0..10}; both children sets
of every node bounded with LB1 and full-pair LB2 (190 machine pairs).  The
metric is bounded children per second (every child gets both bounds).

Native arm (default): the batch is resident in HBM; each step is one launch of
the bounding kernel through pfsp_bound_batch_dev; L2 is flushed (a 256 MiB
write) before every step, outside the timed events.  `e2e` repeats the
measurement through the host-pointer entry point pfsp_bound_batch with pinned
host buffers (host-to-device copy of the nodes and device-to-host copy of both
bound arrays inside the timed region).

Reference arm (--impl reference): the CPU oracle (oracle/) on the host cores,
each step a bounded sample of the same batch.

Multi-GPU (torchrun, one rank per GPU): every rank bounds its own batch (weak
scaling); the only collectives are a barrier and a max of the timings.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_JOBS, M_MACH, N_NODES, SEED, DMAX = 20, 20, 4194304, 2020, 10
WORKLOAD = "pfsp-bound-20x20-4M"
METRIC = "bounded children/s (LB1 + full-pair LB2)"
UNIT = "children/s"
L2_FLUSH_BYTES = 256 << 20
LEARNED_SLOT_CHECKS = None  # learned solver's slot checks: learned.slot_checks_for(m)
REDUCE_UB = 1500  # exclusive incumbent of the reduce mode's survivor masks (near the batch's median LB2)
# INT32 ALU lanes per SM per clock on sm_103a (add, min/max, logic; measured
# at 127.9 IMNMX thread-instructions per SM per clock)
INT32_LANES_PER_SM_CLK = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--nodes", type=int, default=N_NODES)
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="timed end-to-end steps (default: --steps; 0 skips the end-to-end legs)")
    ap.add_argument("--cpu-sample", type=int, default=1000000, help="nodes in the oracle's timed sample")
    ap.add_argument("--ref-sample", type=int, default=400000,
                    help="nodes the reference arm (the oracle) bounds per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-proof leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-ordering comparison")
    ap.add_argument("--solve-seeds", default="1,2,3,4,5,6,7,8,9,10",
                    help="seeds of the time-to-proof leg (comma separated)")
    return ap.parse_args()


def workload_config(nodes, ws):
    """The workload both arms name in their JSON line (identical dicts)."""
    return {"workload": WORKLOAD, "n": N_JOBS, "m": M_MACH, "nodes_per_gpu": nodes, "seed": SEED,
            "depths": "d1, d2 uniform in 0..%d" % DMAX, "bounds": "LB1+LB2 (190 pairs)",
            "l2": "GPU arm: flushed before every step (256 MiB write, outside the timed events); "
                  "oracle arm: host only",
            "parallelism": "independent batches per GPU" if ws > 1 else "1 GPU"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def algorithmic_ops(n, m, d1, d2):
    """Integer operations the bounding method needs per batch:
    front/back wavefronts 2 per cell; per child and machine 6 (recurrence
    max+add, term add+add, max into the bound, remaining-work subtraction);
    LB2 per (pair, unscheduled job) 13: prefix map 2, suffix map 3, C 2 and
    the pair term of both children 2 x 3."""
    d = d1.astype(np.int64) + d2.astype(np.int64)
    u = n - d
    P = m * (m - 1) // 2
    lb1 = 2 * m * d + 2 * u * m * 6
    lb2 = P * u * 13
    return int((lb1 + lb2).sum())


def pin_to_gpu_cpus(dev_index):
    """Run the host side on the CPUs next to the GPU, so that the pinned buffers of the
    end-to-end leg are allocated in the memory of the socket the GPU is attached to.
    Returns a description, or "default" when the topology is not readable."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev_index)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bus) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return "default"
        os.sched_setaffinity(0, cpus)
        return "cpus %s (local to GPU %s)" % (spec, bus)
    except (OSError, ValueError, AttributeError):
        return "default"


def child_by_child_ops(n, m, d1, d2):
    """The per-parent work of the bounds evaluated child by child, as the
    paper's recurrence states them: LB2 4 ops per (child, pair, unscheduled job
    of the child), 2P u (u - 1) such steps; LB1 4m per child and 2m (d1 + d2)
    per parent.  This design evaluates the same values with the O(P u)
    composition counted by algorithmic_ops."""
    d = d1.astype(np.int64) + d2.astype(np.int64)
    u = n - d
    P = m * (m - 1) // 2
    return int((4 * 2 * P * u * np.maximum(u - 1, 0) + 4 * m * 2 * u + 2 * m * d).sum())


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2012_09511_gb300", "csrc")
    for f in ("bound_device.cuh", "bound_kernel.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_summary():
    """The committed ncu summary of the bounding kernel (DRAM bytes per launch,
    pipe and issue utilisation), if it was taken on the current kernel source;
    otherwise None."""
    path = os.path.join(ROOT, "profiles", "bound_kernel_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return t


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(p, perm, d1, d2, sample, total=None, single=0):
    """The oracle as it stands, on the host cores, over a bounded sample of the batch (the
    first `sample` of its `total` nodes; the node generator is counter-based, so a shorter
    draw is a prefix of the full batch); with single > 0 also on one thread over the first
    `single` nodes."""
    import oracle as orc
    cores = len(os.sched_getaffinity(0)) or 1

    def run(k, threads):
        t = time.perf_counter()
        orc.children_bounds_batch(p, perm[:k], d1[:k], d2[:k], threads=threads)
        dt = time.perf_counter() - t
        children = int(2 * (N_JOBS - d1[:k].astype(np.int64) - d2[:k].astype(np.int64)).sum())
        return children / dt, dt

    k = min(sample, len(d1))
    value, dt = run(k, cores)
    out = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
           "sample": "first %d of the %d nodes, LB1 + LB2 from scratch per child, %.1f s" % (
               k, total or len(d1), dt)}
    if single > 0:
        ks = min(single, len(d1))
        v1, dt1 = run(ks, 1)
        out["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1, "seconds": dt1,
                                "sample": "first %d nodes on one thread" % ks}
    return out


def solve_leg(pfsp, seeds=range(1, 11)):
    """Time-to-proof of the exact-solve workload (n = 20, m = 10, LB2): each seed
    solved in proof mode with the incumbent at the oracle's optimum (fixed tree;
    counts checked against the oracle's), and from its NEH schedule."""
    from paper_2012_09511_gb300 import inputs
    path = os.path.join(ROOT, "tests", "golden", "solve_20x10_lb2.json")
    with open(path) as f:
        gold = {r["seed"]: r for r in json.load(f)["results"]}
    per, tot_proof, tot_find, tot_nodes, exact = [], 0.0, 0.0, 0, True
    for seed in seeds:
        g = gold[seed]
        inst = pfsp.pfsp_load_instance(inputs.make_instance(20, 10, seed))
        pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB2, init_ub=g["optimum"])  # warm
        r = pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB2, init_ub=g["optimum"])
        f = pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB2)
        ok = (r["decomposed"] == g["proof_decomposed"] and f["cmax"] == g["optimum"]
              and r["outcome"] == pfsp.PFSP_PROVEN_NO_BETTER)
        exact &= ok
        per.append({"seed": seed, "proof_s": r["kernel_seconds"], "nodes": r["decomposed"],
                    "find_s": f["kernel_seconds"], "optimum": f["cmax"], "exact": ok})
        tot_proof += r["kernel_seconds"]
        tot_find += f["kernel_seconds"]
        tot_nodes += r["decomposed"]
    return {"workload": "n=20 m=10 uniform[1,99] seeds %s, LB2 + MinMin, proof mode at the optimum" % (
                ",".join(str(x) for x in seeds)),
            "time_to_proof_s": tot_proof, "time_to_optimum_from_neh_s": tot_find,
            "decomposed_nodes": tot_nodes, "decomposed_nodes_per_s": tot_nodes / max(tot_proof, 1e-9),
            "counts_and_optima_match_oracle": bool(exact), "per_seed": per,
            "oracle_proof_s_single_thread": sum(gold[s]["oracle_proof_seconds"] for s in seeds),
            "branching_rules": rules_leg(pfsp, gold, seeds),
            "heuristic_threads": heuristic_leg(pfsp, gold, seeds),
            "lb1_minht": minht_leg(pfsp),
            "lb1_30x15_rate": lb1_rate_leg(pfsp)}


def lb1_rate_leg(pfsp, seeds=(1, 2, 3), node_limit=20_000_000):
    """Decomposed nodes per second of the explorer pool with LB1 and MinMin on 30-job,
    15-machine instances (the size and bound of the paper's single-GPU runs on VFR 30x15
    instances, which are not available here: seeded uniform [1, 99] stand-ins), from the
    NEH incumbent, stopped at a node limit."""
    from paper_2012_09511_gb300 import inputs
    nodes, secs = 0, 0.0
    for seed in seeds:
        inst = pfsp.pfsp_load_instance(inputs.make_instance(30, 15, 3000 + seed))
        r = pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB1, node_limit=node_limit)
        nodes += r["decomposed"]
        secs += r["kernel_seconds"]
    return {"workload": "n=30 m=15 uniform[1,99] seeds 3001-3003, LB1 + MinMin from NEH, %d-node limit each" % node_limit,
            "decomposed_nodes": nodes, "kernel_s": secs, "decomposed_nodes_per_s": nodes / max(secs, 1e-9)}


def minht_leg(pfsp):
    """LB1 proofs at the optimum with and without the heads and tails refinement
    (pfsp_options.lb1_minht), node counts checked against tests/golden/solve_lb1_minht.json."""
    from paper_2012_09511_gb300 import inputs
    with open(os.path.join(ROOT, "tests", "golden", "solve_lb1_minht.json")) as f:
        cases = json.load(f)["results"]
    out = {"workload": "LB1 proofs of %d instances (n, m, seed) = %s" % (
        len(cases), ", ".join("(%d,%d,%d)" % (c["n"], c["m"], c["seed"]) for c in cases))}
    for name, flag in (("plain", 0), ("minht", 1)):
        t = 0.0
        nodes, exact = 0, True
        for c in cases:
            inst = pfsp.pfsp_load_instance(inputs.make_instance(c["n"], c["m"], c["seed"]))
            pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB1, init_ub=c["optimum"], lb1_minht=flag)  # warm
            r = pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB1, init_ub=c["optimum"], lb1_minht=flag)
            exact &= r["decomposed"] == c[name]["decomposed"] and r["outcome"] == pfsp.PFSP_PROVEN_NO_BETTER
            t += r["kernel_seconds"]
            nodes += r["decomposed"]
        out[name] = {"time_to_proof_s": t, "decomposed_nodes": nodes, "counts_match_oracle": bool(exact)}
    return out


def heuristic_leg(pfsp, gold, seeds, threads=4):
    """Finding mode from NEH with and without the host heuristic threads (Section 4.2):
    device time and wall time to the proven optimum, nodes decomposed, and what the threads
    contributed.  Node counts differ between runs here, so only the optima are checked."""
    from paper_2012_09511_gb300 import inputs
    out = {"threads": threads, "kinds": "with: iterated greedy; with_beam: beam search below the promoted "
                                          "explorer nodes; with_both: half the threads each"}
    for name, t, kind in (("without", 0, 0), ("with", threads, 0), ("with_beam", threads, 1),
                          ("with_both", threads, 2)):
        kern = wall = 0.0
        nodes, improved, exact = 0, 0, True
        for seed in seeds:
            g = gold[seed]
            inst = pfsp.pfsp_load_instance(inputs.make_instance(20, 10, seed))
            r = pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB2, heuristic_threads=t, heuristic_seed=seed,
                                heuristic_kind=kind)
            exact &= r["cmax"] == g["optimum"] and r["outcome"] == pfsp.PFSP_OPTIMAL
            kern += r["kernel_seconds"]
            wall += r["seconds"]
            nodes += r["decomposed"]
            improved += int(r["heuristic_improvements"] > 0)
        out[name] = {"time_to_optimum_kernel_s": kern, "time_to_optimum_wall_s": wall, "decomposed_nodes": nodes,
                     "seeds_improved_by_threads": improved, "optima_match_oracle": bool(exact)}
    return out


def rules_leg(pfsp, gold, seeds):
    """The same seeds under the other branching rules (capped MinMin, MinBranch, MinSum):
    time-to-proof at the optimum (counts checked against the oracle's where recorded) and
    time to the optimum from NEH."""
    from paper_2012_09511_gb300 import inputs
    path = os.path.join(ROOT, "tests", "golden", "solve_20x10_rules.json")
    rg = {}
    if os.path.exists(path):
        with open(path) as f:
            rg = {r["seed"]: r for r in json.load(f)["results"]}
    out = {}
    for name, rule in (("minmin_capped", pfsp.PFSP_MINMIN_CAPPED), ("minbranch", pfsp.PFSP_MINBRANCH),
                       ("minsum", pfsp.PFSP_MINSUM)):
        proof = find = 0.0
        nodes, exact, checked = 0, True, 0
        for seed in seeds:
            g = gold[seed]
            inst = pfsp.pfsp_load_instance(inputs.make_instance(20, 10, seed))
            r = pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB2, init_ub=g["optimum"], branching=rule)
            f = pfsp.pfsp_solve(inst, bound=pfsp.PFSP_LB2, branching=rule)
            want = g["proof_capped_decomposed"] if name == "minmin_capped" else \
                rg.get(seed, {}).get(name, {}).get("decomposed")
            ok = f["cmax"] == g["optimum"] and r["outcome"] == pfsp.PFSP_PROVEN_NO_BETTER
            if want is not None:
                ok &= r["decomposed"] == want
                checked += 1
            exact &= ok
            proof += r["kernel_seconds"]
            find += f["kernel_seconds"]
            nodes += r["decomposed"]
        out[name] = {"time_to_proof_s": proof, "time_to_optimum_from_neh_s": find, "decomposed_nodes": nodes,
                     "counts_checked": checked, "counts_and_optima_match_oracle": bool(exact)}
    return out


def batch_leg(pfsp):
    """The uneven batch: 256 independent instances (n in 12..20, m in {5, 10, 20},
    times uniform in [1, 99]) solved from NEH in one persistent launch recorded in a
    CUDA graph, with the autotuner's launch parameters; optima checked against the
    oracle's where it finished."""
    from paper_2012_09511_gb300 import inputs
    path = os.path.join(ROOT, "tests", "golden", "batch256_lb2.json")
    with open(path) as f:
        gold = {r["i"]: r for r in json.load(f)["results"]}
    ps = [inputs.make_instance(*inputs.batch_instance_shape(i), 1000 + i) for i in range(256)]
    insts = [pfsp.pfsp_load_instance(p) for p in ps]
    t = time.perf_counter()
    tuned = pfsp.pfsp_autotune_batch(insts, pfsp.pfsp_default_options(bound=pfsp.PFSP_LB2), sample=32)
    tune_s = time.perf_counter() - t
    pfsp.pfsp_solve_batch(insts, tuned)  # warm
    t = time.perf_counter()
    r = pfsp.pfsp_solve_batch(insts, tuned)
    wall = time.perf_counter() - t
    st = r["stats"]
    checked = [i for i in range(256) if "optimum" in gold.get(i, {})]
    match = all(int(r["cmax"][i]) == gold[i]["optimum"] for i in checked)
    return {"workload": "256 instances, n = 12 + (h_i mod 9), m in {5, 10, 20}, seeds 1000-1255, LB2 + MinMin, "
                        "from NEH, one launch",
            "kernel_s": st["kernel_seconds"], "wall_s": wall, "decomposed_nodes": st["decomposed"],
            "decomposed_nodes_per_s": st["decomposed"] / max(st["kernel_seconds"], 1e-9),
            "all_optimal": bool((r["outcomes"] == pfsp.PFSP_OPTIMAL).all()),
            "optima_checked_against_oracle": len(checked), "optima_match_oracle": bool(match),
            "autotuned": {"warps_per_sm": tuned.warps_per_sm, "slot_warps": tuned.slot_warps,
                          "instance_slots": st["explorers"] // max(tuned.slot_warps, 1),
                          "check_every": tuned.check_every,
                          "min_steal": tuned.min_steal, "tuning_s": tune_s}}


def learned_leg(pfsp):
    """Learned solver vs the plain full-pair LB2 solver, proving known optima:
    n = 30, m = 10 (the ten seeds of learned.SEEDS_30X10, whose plain proofs
    take at least 50 ms each), n = 50, m = 5 (seeds 101-110; these proofs take
    well under a millisecond), n = 18 and 20, m = 20 (seeds 101-103, where the
    pairs fill six 32-pair slots and the slot checks are on).  Both under capped MinMin (identical trees,
    counts checked equal) and under the paper's MinMin (node inflation
    reported); kernel and wall times are the median of three solves.  The
    m-machine networks are trained on the GPU on the solver's own traces of
    other instances with the same m."""
    from paper_2012_09511_gb300 import inputs, learned
    mlps, training = {}, {}
    for m in (5, 10, 20):
        t = time.perf_counter()
        nt = 16 if m == 20 else 20  # 20-machine traces from 16-job instances, which solve in milliseconds
        mlps[m], info = learned.train_network(pfsp, m, [inputs.make_instance(nt, m, s) for s in range(1, 11)],
                                              nodes_per_instance=3000 if m == 20 else 4000)
        info["seconds"] = time.perf_counter() - t
        training["m=%d" % m] = info
    cases = {"30x10": (30, 10, learned.SEEDS_30X10), "50x5": (50, 5, range(101, 111)),
             "18x20": (18, 20, range(101, 104)), "20x20": (20, 20, range(101, 104))}
    rules = (("minmin_capped", pfsp.PFSP_MINMIN_CAPPED), ("minmin", pfsp.PFSP_MINMIN))
    rep = learned.compare_proofs(pfsp, cases, mlps, rules=rules, reps=3, slot_checks=LEARNED_SLOT_CHECKS)
    find = learned.compare_finding(pfsp, 30, 10, learned.SEEDS_30X10, mlps[10], rule=pfsp.PFSP_MINMIN)
    for name, r in rep.items():
        c = r.get("minmin_capped")
        if c:
            c["counts_equal_plain"] = c["decomposed"]["learned"] == c["decomposed"]["plain"]
    return {"training": training,
            "learned_solver": "network pair order (root's children) + early exit per child%s" % (
                " + slot checks" if LEARNED_SLOT_CHECKS else
                " + slot checks from four 32-pair slots (m >= 15)" if LEARNED_SLOT_CHECKS is None else ""),
            "ablations": "early_exit_index_order: the same early exit, pairs in index order; "
                         "pair_subset: LB2 over the network's top half of the 32-pair slots (weaker bound)",
            "proofs": rep,
            "finding_30x10": dict(find, workload="30 x 10 seeds of the proofs, from NEH to the proven optimum, "
                                                 "MinMin, one solve each")}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2012_09511_gb300 import inputs
    p = inputs.make_instance(N_JOBS, M_MACH, SEED)
    sample = min(args.ref_sample, args.nodes)
    perm, d1, d2 = inputs.random_nodes(N_JOBS, sample, seed=SEED)
    for _ in range(args.warmup):
        cpu_baseline(p, perm, d1, d2, min(2000, sample))
    times = []
    for _ in range(args.steps):
        r = cpu_baseline(p, perm, d1, d2, sample, total=args.nodes)
        times.append(r)
    # the rate over all steps: children bounded / seconds, summed
    value = sum(t["value"] * t["seconds"] for t in times) / max(sum(t["seconds"] for t in times), 1e-9)
    step_ms = statistics.mean([t["seconds"] for t in times]) * 1e3
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int32", "data": "synthetic", "impl": "reference",
           "config": workload_config(args.nodes, 1),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": times[0]["cores"], "kind": "oracle",
                            "sample": times[0]["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_native(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    host_cpus = pin_to_gpu_cpus(local)
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import inputs, pfsp, shard

    n, m, N = N_JOBS, M_MACH, args.nodes
    p = inputs.make_instance(n, m, SEED)
    perm, d1, d2 = inputs.random_nodes(n, N, seed=shard.rank_seed(SEED, rank), dmax=DMAX)
    children = int(2 * (n - d1.astype(np.int64) - d2.astype(np.int64)).sum())
    ops = algorithmic_ops(n, m, d1, d2)
    inst = pfsp.pfsp_load_instance(p)
    tp = torch.from_numpy(perm).to(dev)
    t1 = torch.from_numpy(d1).to(dev)
    t2 = torch.from_numpy(d2).to(dev)
    o1 = torch.empty((N, 2, n), dtype=torch.int32, device=dev)
    o2 = torch.empty_like(o1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step():
        pfsp.pfsp_bound_batch_dev(inst, pfsp.PFSP_LB1 | pfsp.PFSP_LB2, N, tp.data_ptr(), t1.data_ptr(),
                                  t2.data_ptr(), o1.data_ptr(), o2.data_ptr(), sh)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = vis.split(",")[local].strip() if vis else str(local)
    sampler = ClockSampler(smi_index)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    launch_ms = ms / args.steps
    value, slowest_s, _ = shard.whole_job_rate(ms * 1e-3, children * args.steps, device=dev)

    # end to end through the host-pointer entry point, pinned host buffers
    hp = torch.from_numpy(perm).pin_memory()
    hd1 = torch.from_numpy(d1).pin_memory()
    hd2 = torch.from_numpy(d2).pin_memory()
    h1 = torch.empty((N, 2, n), dtype=torch.int32).pin_memory()
    h2 = torch.empty((N, 2, n), dtype=torch.int32).pin_memory()
    args_np = (hp.numpy(), hd1.numpy(), hd2.numpy())
    e2e_steps = args.steps if args.e2e_steps < 0 else args.e2e_steps

    def timed_steps(call):
        # W untimed calls (the first allocates the library's staging scratch),
        # then the same number of timed steps as the device leg; per-step wall
        # times are kept, the rate is taken over their sum (the mean step)
        if e2e_steps > 0:
            for _ in range(max(args.warmup, 1)):
                call()
        if ws > 1:
            dist.barrier()
        ts = []
        # no garbage collection pass in the middle of a timed step
        gc_was = gc.isenabled()
        gc.disable()
        try:
            for _ in range(e2e_steps):
                t0 = time.perf_counter()
                call()
                ts.append(time.perf_counter() - t0)
        finally:
            if gc_was:
                gc.enable()
        return ts

    def rates(ts):
        mean, _, _ = shard.whole_job_rate(max(sum(ts), 1e-9), children * len(ts), device=dev)
        med, _, _ = shard.whole_job_rate(max(statistics.median(ts), 1e-9) if ts else 1e-9, children if ts else 0,
                                         device=dev)
        return mean, med

    e2e_ts = timed_steps(lambda: pfsp.pfsp_bound_batch(inst, 3, *args_np, lb1_out=h1.numpy(), lb2_out=h2.numpy()))
    e2e_value, e2e_median = rates(e2e_ts)

    # reduce mode: the same nodes and bounds (LB2, the solver's), one
    # 48-byte summary per parent instead of the bound arrays
    ub_reduce = REDUCE_UB
    so = torch.empty(N * pfsp.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev)

    def rstep():
        pfsp.pfsp_bound_reduce_dev(inst, pfsp.PFSP_LB2, N, tp.data_ptr(), t1.data_ptr(), t2.data_ptr(),
                                   ub_reduce, so.data_ptr(), sh)

    for _ in range(args.warmup):
        flush.fill_(1)
        rstep()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    revs = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rstep()
        e1.record(stream)
        revs.append((e0, e1))
    torch.cuda.synchronize()
    r_ms = sum(a.elapsed_time(b) for a, b in revs)
    r_value, _, _ = shard.whole_job_rate(r_ms * 1e-3, children * args.steps, device=dev)
    hs = np.empty(N, dtype=pfsp.SUMMARY_DTYPE)
    hs_pin = torch.from_numpy(hs.view(np.uint8)).pin_memory()
    hs = hs_pin.numpy().view(pfsp.SUMMARY_DTYPE)
    r_ts = timed_steps(lambda: pfsp.pfsp_bound_reduce(inst, pfsp.PFSP_LB2, *args_np, ub_reduce, out=hs))
    r_e2e_value, r_e2e_median = rates(r_ts)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_ops = nsm * INT32_LANES_PER_SM_CLK * sm_max * 1e6
    achieved = ops / (launch_ms * 1e-3)
    ncu = ncu_summary()
    traffic = ncu.get("dram_bytes_per_launch_full") if ncu else None
    cbc_ops = child_by_child_ops(n, m, d1, d2)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": slowest_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(N, ws),
        "host_cpus": host_cpus,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
                     "frac": achieved / peak_ops, "traffic": traffic,
                     "peak_source": "%d SMs x %d INT32 lanes/clk x %.0f MHz (max SM clock)" % (
                         nsm, INT32_LANES_PER_SM_CLK, sm_max),
                     "ops_per_launch": ops, "kernel_ms": launch_ms,
                     "child_by_child_ops_per_launch": cbc_ops,
                     "child_by_child_frac": cbc_ops / (launch_ms * 1e-3) / peak_ops,
                     "ncu_utilisation": {k: ncu[k] for k in ("issue_active_pct", "alu_pipe_pct", "fma_pipe_inst_pct",
                                                             "fmaheavy_cycles_pct", "lsu_pipe_pct") if k in ncu}
                     if ncu else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(N * (n + 2)),
                "d2h_bytes_per_step": int(2 * N * 2 * n * 4),
                "statistic": "mean of %d steps through pfsp_bound_batch (after %d untimed)" % (
                    len(e2e_ts), max(args.warmup, 1)), "median_value": e2e_median,
                "step_ms": [round(t * 1e3, 2) for t in e2e_ts]},
        "reduce": {"value": r_value, "unit": UNIT, "ms_per_step": r_ms / args.steps,
                   "mode": "LB2 summarised per parent and direction (least bound, count, sum, survivors "
                           "below %d), 48 bytes per parent" % REDUCE_UB,
                   "e2e": {"value": r_e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(N * (n + 2)),
                           "d2h_bytes_per_step": int(N * 48), "median_value": r_e2e_median,
                           "step_ms": [round(t * 1e3, 2) for t in r_ts]}},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(p, perm, d1, d2, args.cpu_sample, total=N, single=20000)
    if not args.no_solve and ws == 1:
        out["solve"] = solve_leg(pfsp, seeds=[int(x) for x in args.solve_seeds.split(",") if x])
    if not args.no_solve and ws == 1:
        out["batch"] = batch_leg(pfsp)
    if not args.no_learned and ws == 1:
        out["learned"] = learned_leg(pfsp)
    out["summary"] = summary_of(out)  # last key: the end of the line carries the other legs' headlines
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def summary_of(out):
    """The headline figures of every leg, compact, for the end of the line."""
    def r(x, nd=4):
        return None if x is None else round(float(x), nd)

    sm = {"bounding": {"children_per_s": r(out["value"] / 1e9, 3), "unit": "1e9 children/s",
                       "kernel_ms": r(out["roofline"]["kernel_ms"], 3), "roofline_frac": r(out["roofline"]["frac"]),
                       "e2e_children_per_s": r(out["e2e"]["value"] / 1e9, 3)}}
    if "reduce" in out:
        sm["bounding"]["reduce_children_per_s"] = r(out["reduce"]["value"] / 1e9, 3)
    if "solve" in out:
        s = out["solve"]
        sm["time_to_proof_20x10"] = {"seconds": r(s["time_to_proof_s"], 5), "nodes": s["decomposed_nodes"],
                                     "nodes_per_s": r(s["decomposed_nodes_per_s"] / 1e6, 1), "unit": "1e6 nodes/s",
                                     "counts_match_oracle": s["counts_and_optima_match_oracle"]}
        if "lb1_30x15_rate" in s:
            sm["lb1_30x15_nodes_per_s"] = r(s["lb1_30x15_rate"]["decomposed_nodes_per_s"] / 1e6, 1)
    if "batch" in out:
        b = out["batch"]
        sm["batch_256"] = {"kernel_s": r(b["kernel_s"], 3), "nodes_per_s": r(b["decomposed_nodes_per_s"] / 1e6, 1),
                           "all_optimal": b["all_optimal"], "optima_checked": b["optima_checked_against_oracle"],
                           "optima_match_oracle": b["optima_match_oracle"]}
    if "learned" in out:
        lp = out["learned"].get("proofs", {})
        sm["learned_vs_plain"] = {
            shape: {rule: {"speedup_kernel": r(v[rule]["speedup_kernel"], 3),
                           "node_ratio": r(v[rule]["node_ratio_learned_over_plain"], 4)}
                    for rule in ("minmin_capped", "minmin") if rule in v}
            for shape, v in lp.items()}
    return sm


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
