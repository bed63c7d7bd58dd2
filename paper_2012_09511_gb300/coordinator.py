"""Work-unit coordinator for several explorer pools (Section 4.1, Algorithm 1).

The paper's coordinator hands out work units -- finite unions of disjoint
half-open intervals [a, b) of leaf indices of the permutation tree, numbered
0 .. n!-1 in lexicographic order (Section 2.6, Eq. 2) -- to worker processes
that each drive one GPU, and keeps a copy of every unit it gave out.  When a
worker reports its unit (a checkpoint message), the coordinator intersects it
with the copy (Eq. 3 and 4); an empty result means the worker is idle, and it
then receives unassigned intervals or the right halves of the first intervals
of the largest unit (work-unit division).  The victim learns of the theft at
its next report, when the intersection returns its shortened unit.

Here a worker is an explorer pool on one GPU, run in segments with
pfsp_solve_resumable: its unit travels as the library's checkpoint bytes.
Intervals are Python integers (the paper uses GMP decimal numbers) and are
converted to factoradic digits only to build those bytes.  Each interval
carries the start level the pool needs to resume without decomposing a node
twice (-1 for an interval that starts at an arbitrary leaf).

Everything here is host-side bookkeeping; all searching runs in the
library's kernels.  run_ranks() drives N workers, one per rank of a
torch.distributed process group, in bulk-synchronous rounds.
"""
from __future__ import annotations

import struct
from math import factorial

CKPT_MAGIC = b"PFSPCKP1"
# magic, n, m, bound, branching, cap, ub, count, have_perm, best_perm[64]
_HEADER = struct.Struct("<8s8i64s")
RECORD_BYTES = 132


# ------------------------------------------------------- factoradic numbers ---

def to_factoradic(n: int, x: int) -> list:
    """Digits d[0..n-1] of x in [0, n!), d[i] in [0, n - i): x = sum d[i] (n-1-i)!."""
    if not 0 <= x < factorial(n):
        raise ValueError("leaf index out of range")
    d = [0] * n
    for i in range(n - 1, -1, -1):
        r = n - i
        d[i] = x % r
        x //= r
    return d


def from_factoradic(d) -> int:
    n = len(d)
    x = 0
    for i in range(n):
        x = x * (n - i) + int(d[i])
    return x


# ------------------------------------------------------- checkpoint bytes -----

def pack_checkpoint(n, m, bound, branching, cap, ub, intervals, best_perm=None) -> bytes:
    """Checkpoint bytes (the layout pfsp_solve_resumable reads) holding the given
    intervals: a list of (a, b, level), 0 <= a < b <= n!, level -1 or the start
    level recorded by the library."""
    nf = factorial(n)
    perm = bytes(best_perm) + b"\xff" * (64 - len(best_perm)) if best_perm is not None else b"\xff" * 64
    out = [_HEADER.pack(CKPT_MAGIC, n, m, bound, branching, cap, ub, len(intervals), int(best_perm is not None),
                        perm)]
    for a, b, lvl in intervals:
        if not 0 <= a < b <= nf:
            raise ValueError("bad interval [%d, %d)" % (a, b))
        rec = bytearray(RECORD_BYTES)
        rec[0] = 1
        rec[1] = 0xFF if lvl < 0 else lvl
        rec[2] = 1 if b == nf else 0
        rec[4:4 + n] = bytes(to_factoradic(n, a))
        if b < nf:
            rec[68:68 + n] = bytes(to_factoradic(n, b))
        out.append(bytes(rec))
    return b"".join(out)


def unpack_checkpoint(buf: bytes):
    """(header dict, [(a, b, level), ...]) of checkpoint bytes."""
    magic, n, m, bound, branching, cap, ub, count, have_perm, perm = _HEADER.unpack_from(buf, 0)
    if magic != CKPT_MAGIC:
        raise ValueError("not a pfsp checkpoint")
    nf = factorial(n)
    iv = []
    o = _HEADER.size
    for _ in range(count):
        rec = buf[o:o + RECORD_BYTES]
        o += RECORD_BYTES
        a = from_factoradic(rec[4:4 + n])
        b = nf if rec[2] else from_factoradic(rec[68:68 + n])
        iv.append((a, b, -1 if rec[1] == 0xFF else rec[1]))
    head = dict(n=n, m=m, bound=bound, branching=branching, cap=cap, ub=ub,
                best_perm=list(perm[:n]) if have_perm else None)
    return head, sorted(iv)


# ------------------------------------------------------- work-unit algebra ----

def size(unit) -> int:
    """||W|| = sum of the interval lengths."""
    return sum(iv[1] - iv[0] for iv in unit)


def intersect(w, c):
    """W cap C for two sorted lists of disjoint intervals (Eq. 3 and 4), in one
    merge pass.  Intervals of w may carry a level (third item); it is kept when
    the start of the interval is unchanged, else it becomes -1."""
    out, i, j = [], 0, 0
    while i < len(w) and j < len(c):
        a = max(w[i][0], c[j][0])
        b = min(w[i][1], c[j][1])
        if a < b:
            lvl = w[i][2] if len(w[i]) > 2 and a == w[i][0] else -1
            out.append((a, b, lvl))
        if w[i][1] < c[j][1]:
            i += 1
        else:
            j += 1
    return out


def split_even(unit, parts: int):
    """Cut every interval of a fresh unit into up to `parts` pieces of equal
    length (pieces start at arbitrary leaves, so their level is -1)."""
    out = []
    for a, b, lvl in unit:
        k = max(1, min(parts, b - a))
        cuts = [a + (b - a) * t // k for t in range(k + 1)]
        for t in range(k):
            if cuts[t] < cuts[t + 1]:
                out.append((cuts[t], cuts[t + 1], lvl if t == 0 else -1))
    return out


class Coordinator:
    """The coordinator of Algorithm 1 for workers identified by small integers.

    W_unassigned starts as [0, n!) (or the given intervals); `units[i]` is the
    copy of worker i's unit; `modified` flags the copies split since their
    worker's last report."""

    def __init__(self, n: int, initial=None, ub: int = 2**31 - 1, best_perm=None):
        self.n = n
        self.unassigned = [(a, b) for a, b in (initial or [(0, factorial(n))])]
        self.units = {}
        self.modified = set()
        self.ub = ub
        self.best_perm = best_perm
        self.steals = 0

    def try_improve(self, ub: int, perm=None) -> None:
        if ub < self.ub:
            self.ub = ub
            self.best_perm = perm

    def checkpoint(self, wid: int, unit, kmax: int):
        """WorkerCheckpoint: intersect the reported unit with the copy; when
        that is empty, steal for the worker.  Returns the worker's new unit (a
        sorted list of (a, b, level)); empty when no work is left anywhere."""
        # a unit only shrinks from the left on the worker's side, so without a
        # theft since the last report the intersection is the report itself
        if wid in self.modified:
            tmp = intersect(sorted(unit), self.units.get(wid, []))
        else:
            tmp = [iv if len(iv) > 2 else (iv[0], iv[1], -1) for iv in sorted(unit)]
        self.modified.discard(wid)
        if not tmp:
            tmp = self._steal(wid, kmax)
        if tmp:
            self.units[wid] = [(a, b) for a, b, _ in tmp]
        else:
            self.units.pop(wid, None)
        return tmp

    def round(self, reports: dict, kmax: int) -> dict:
        """Bulk-synchronous form of WorkerCheckpoint for all workers at once:
        every report is intersected with its copy first, then every idle
        worker steals, and only then are the answers formed, so that a victim's
        answer already excludes the halves taken from it.  In the asynchronous
        form (checkpoint()) a victim keeps exploring its old unit until its next
        report and may decompose part of a stolen half twice; here every leaf
        belongs to exactly one worker in every round."""
        tmp = {}
        for wid, unit in reports.items():
            if wid in self.modified:
                tmp[wid] = intersect(sorted(unit), self.units.get(wid, []))
            else:
                tmp[wid] = [iv if len(iv) > 2 else (iv[0], iv[1], -1) for iv in sorted(unit)]
            self.modified.discard(wid)
            if tmp[wid]:
                self.units[wid] = [(a, b) for a, b, _ in tmp[wid]]
            else:
                self.units.pop(wid, None)
        for wid in reports:
            if not tmp[wid]:
                tmp[wid] = self._steal(wid, kmax)
                if tmp[wid]:
                    self.units[wid] = [(a, b) for a, b, _ in tmp[wid]]
        out = {}
        for wid in reports:
            if wid in self.modified:  # robbed in this round
                out[wid] = intersect(tmp[wid], self.units.get(wid, []))
                self.modified.discard(wid)
            else:
                out[wid] = tmp[wid]
        return out

    def _steal(self, wid: int, kmax: int):
        if self.unassigned:
            take, self.unassigned = self.unassigned[:kmax], self.unassigned[kmax:]
            return [(a, b, -1) for a, b in take]
        # work-unit division: right halves of the first min(kmax, K_v)
        # splittable intervals of the largest unit
        victims = [(size(u), v) for v, u in self.units.items() if v != wid]
        if not victims:
            return []
        sz, v = max(victims)
        if sz < 2:
            return []
        unit, new, kept, taken = self.units[v], [], [], 0
        for a, b in unit:
            if taken < kmax and b - a >= 2:
                mid = (a + b) // 2
                kept.append((a, mid))
                new.append((mid, b, -1))
                taken += 1
            else:
                kept.append((a, b))
        self.units[v] = kept
        self.modified.add(v)
        self.steals += 1
        return new

    def done(self) -> bool:
        return not self.unassigned and not any(self.units.values())


# ------------------------------------------------------- GPU worker -----------

class PoolWorker:
    """One explorer pool (one GPU) working on its unit in segments of at most
    `node_limit` counted decompositions."""

    def __init__(self, pfsp, inst, bound, branching=0, cap=None, learned=0, node_limit=100000, kmax=512):
        self.pfsp, self.inst = pfsp, inst
        self.bound, self.branching, self.learned = bound, branching, learned
        self.cap = cap
        self.node_limit, self.kmax = node_limit, kmax
        self.unit = []
        self.counts = {"decomposed": 0, "bounded_children": 0, "pruned": 0, "leaves": 0}
        self.segments = 0

    def run(self, unit, ub, best_perm=None):
        """Explore `unit` (sorted (a, b, level) list) for one segment from the
        incumbent ub; returns (remaining unit, incumbent, schedule or None)."""
        if not unit:
            return [], ub, None
        n, m = self.inst.n, self.inst.m
        if len(unit) < self.kmax // 4 and all(lvl < 0 for _, _, lvl in unit):
            unit = split_even(unit, self.kmax // (4 * len(unit)))
        ck = pack_checkpoint(n, m, self.bound, self.branching, self.cap, ub, unit[:self.kmax], best_perm)
        r = self.pfsp.pfsp_solve_resumable(self.inst, resume=ck, bound=self.bound, branching=self.branching,
                                           learned=self.learned, node_limit=self.node_limit)
        self.segments += 1
        for k in self.counts:
            self.counts[k] += r[k]
        rest = unit[self.kmax:]
        left = unpack_checkpoint(r["checkpoint"])[1] if r["checkpoint"] else []
        perm = [int(x) for x in r["perm"]] if r["perm"][0] >= 0 else None
        return sorted(left + rest), r["cmax"], perm


def solve_with_workers(workers, coord: Coordinator, max_rounds=100000):
    """Bulk-synchronous rounds on one process: every worker reports, the
    coordinator answers (Algorithm 1), every worker runs one segment.  Used to
    drive several pools in turn on one GPU, or as the body of run_ranks."""
    reports = {i: [] for i in range(len(workers))}
    for _ in range(max_rounds):
        units = coord.round(reports, min(w.kmax for w in workers))
        if coord.done():
            return coord
        for i, w in enumerate(workers):
            left, ub, perm = w.run(units[i], coord.ub, coord.best_perm)
            coord.try_improve(ub, perm)
            reports[i] = left
    raise RuntimeError("coordinator did not finish within max_rounds")


def run_ranks(worker, coord_factory, group=None, max_rounds=100000):
    """One worker per rank of the default torch.distributed group (gloo for
    host objects): rank 0 also runs the coordinator.  Each round every rank
    sends (its unit, its incumbent, its schedule) to rank 0, rank 0 answers with
    the rank's new unit and the global incumbent, and every rank runs one
    segment.  Returns the coordinator on rank 0 (None elsewhere) and the
    worker's counters."""
    import torch.distributed as dist
    rank, ws = dist.get_rank(group), dist.get_world_size(group)
    coord = coord_factory() if rank == 0 else None
    report = ([], 2**31 - 1, None)
    for _ in range(max_rounds):
        gathered = [None] * ws if rank == 0 else None
        dist.gather_object(report, gathered, dst=0, group=group)
        answers = [None] * ws
        if rank == 0:
            for unit, ub, perm in gathered:
                coord.try_improve(ub, perm)
            units = coord.round({i: gathered[i][0] for i in range(ws)}, worker.kmax)
            stop = coord.done()
            answers = [(units[i], coord.ub, coord.best_perm, stop) for i in range(ws)]
        mine = [None]
        dist.scatter_object_list(mine, answers if rank == 0 else None, src=0, group=group)
        unit, ub, best, stop = mine[0]
        if stop:
            return coord, worker.counts
        left, ub2, perm = worker.run(unit, ub, best)
        report = (left, ub2, perm)
    raise RuntimeError("coordinator did not finish within max_rounds")
