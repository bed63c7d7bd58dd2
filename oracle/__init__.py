"""CPU oracle for the PFSP branch-and-bound hot path (arXiv 2012.09511).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain sequential C library
(`pfsp_oracle.c`) that computes every quantity of the method from its
definition; this module builds it with gcc and marshals numpy arrays through
ctypes.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it; the product package never does, and the two share no code.

Functions and the paper passages they follow:
  makespan / completion ... Eq. 1 (Section 2.1)
  front, back, remain, lb1  Section 2.4, LB1 steps 1-4 (lb1 minht=True: empty
                            heads and tails raised to the least upstream /
                            downstream work of an unscheduled job; not in the
                            paper)
  lb2, johnson ............ Section 2.4 (two-machine bound, Johnson's rule)
  children_bounds ......... Section 2.3 (forward/backward children), 2.4
  minmin .................. Section 2.3 (MinMin branching rule)
  branch_rule ............. Section 2.3 and Table 4 (readings of MinBranch
                            and MinSum, which the paper names only)
  bb_solve ................ Sections 2.2-2.5 (DFS branch-and-bound)
  factoradic_*, midpoint .. Section 2.6 (work units, work stealing)
  ivm_decode .............. Section 2.5 (IVM decoding)
  brute_force, neh ........ exact enumeration; NEH initial upper bound
                            (NEH is not in the paper)
  mlp ..................... learned ordering network (not in the paper),
                            see oracle/mlp_ref.py
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfsp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FWD, BWD = 0, 1
LB1, LB2 = 1, 2
MINHT = 4  # bit of kind / bound: LB1 with the heads and tails refinement (not in the paper)
MINMIN, MINMIN_CAPPED, MINBRANCH, MINSUM = 0, 1, 2, 3
OPTIMAL, PROVEN_NO_BETTER, LIMIT_NODES = 0, 1, 2
INT32_MAX = 2**31 - 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C11, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L = _lib
        L.orc_makespan.restype = ctypes.c_int32
        L.orc_makespan.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p]
        L.orc_completion.restype = None
        L.orc_completion.argtypes = [ctypes.c_int, i32p, i32p, ctypes.c_int, i32p]
        L.orc_front.argtypes = [ctypes.c_int, i32p, i32p, ctypes.c_int, i32p]
        L.orc_back.argtypes = [ctypes.c_int, i32p, i32p, ctypes.c_int, i32p]
        L.orc_remain.argtypes = [ctypes.c_int, ctypes.c_int, i32p, u8p, i32p]
        L.orc_lb1_combine.restype = ctypes.c_int32
        L.orc_lb1_combine.argtypes = [ctypes.c_int, i32p, i32p, i32p]
        for f in (L.orc_lb1, L.orc_lb2, L.orc_lb1_minht):
            f.restype = ctypes.c_int32
            f.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int, i32p, ctypes.c_int]
        L.orc_pair_value.restype = ctypes.c_int32
        L.orc_pair_value.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, ctypes.c_int,
                                     i32p, i32p, i32p, ctypes.c_int]
        L.orc_johnson_lag_order.argtypes = [ctypes.c_int, i32p, i32p, i32p, i32p]
        L.orc_johnson.restype = ctypes.c_int32
        L.orc_johnson.argtypes = [ctypes.c_int, i32p, i32p]
        L.orc_children_bounds.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, u8p,
                                          ctypes.c_int, ctypes.c_int, i32p, i32p]
        L.orc_children_bounds_batch.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int,
                                                ctypes.c_int64, u8p, u8p, u8p, i32p, i32p,
                                                ctypes.c_int]
        L.orc_children_bounds_batch_pairs.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int,
                                                      ctypes.c_int64, u8p, u8p, u8p, i32p, i32p,
                                                      ctypes.c_int, i32p, ctypes.c_int]
        L.orc_bb_solve_pairs.restype = ctypes.c_int
        L.orc_bb_solve_pairs.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int32, ctypes.c_int64, i32p, i32p, i64p, i32p, ctypes.c_int]
        L.orc_minmin.restype = ctypes.c_int
        L.orc_minmin.argtypes = [ctypes.c_int, i32p, i32p, u8p, ctypes.c_int32]
        L.orc_branch_rule.restype = ctypes.c_int
        L.orc_branch_rule.argtypes = [ctypes.c_int, i32p, i32p, u8p, ctypes.c_int, ctypes.c_int32]
        L.orc_bb_solve.restype = ctypes.c_int
        L.orc_bb_solve.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int32, ctypes.c_int64, i32p, i32p, i64p]
        L.orc_brute_force.restype = ctypes.c_int32
        L.orc_brute_force.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p]
        L.orc_neh.restype = ctypes.c_int32
        L.orc_neh.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p]
        L.orc_factoradic_from_decimal.argtypes = [ctypes.c_int, ctypes.c_uint64, i32p]
        L.orc_factoradic_to_decimal.restype = ctypes.c_uint64
        L.orc_factoradic_to_decimal.argtypes = [ctypes.c_int, i32p]
        L.orc_steal_midpoint.restype = ctypes.c_uint64
        L.orc_steal_midpoint.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_ivm_decode.argtypes = [ctypes.c_int, i32p, i32p, i32p, i32p, i32p, i32p]
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _shape(p):
    p = np.asarray(p)
    return p.shape[0], p.shape[1]


def makespan(p, perm) -> int:
    n, m = _shape(p)
    P, pp = _i32(p)
    Q, qp = _i32(perm)
    return int(lib().orc_makespan(n, m, pp, qp))


def completion(p, seq):
    n, m = _shape(p)
    P, pp = _i32(p)
    S, sp = _i32(seq)
    C, cp = _i32(np.zeros(m))
    lib().orc_completion(m, pp, sp, len(S), cp)
    return C


def front(p, sigma1):
    n, m = _shape(p)
    P, pp = _i32(p)
    S, sp = _i32(sigma1 if len(sigma1) else [0])
    F, fp = _i32(np.zeros(m))
    lib().orc_front(m, pp, sp, len(sigma1), fp)
    return F


def back(p, sigma2):
    n, m = _shape(p)
    P, pp = _i32(p)
    S, sp = _i32(sigma2 if len(sigma2) else [0])
    B, bp = _i32(np.zeros(m))
    lib().orc_back(m, pp, sp, len(sigma2), bp)
    return B


def remain(p, unscheduled):
    n, m = _shape(p)
    P, pp = _i32(p)
    un = np.zeros(n, dtype=np.uint8)
    un[list(unscheduled)] = 1
    U, up = _u8(un)
    R, rp = _i32(np.zeros(m))
    lib().orc_remain(n, m, pp, up, rp)
    return R


def lb1_combine(front_, remain_, back_) -> int:
    F, fp = _i32(front_)
    R, rp = _i32(remain_)
    B, bp = _i32(back_)
    return int(lib().orc_lb1_combine(len(F), fp, rp, bp))


def _bound(fn, p, sigma1, sigma2):
    n, m = _shape(p)
    P, pp = _i32(p)
    S1, s1 = _i32(list(sigma1) or [0])
    S2, s2 = _i32(list(sigma2) or [0])
    return int(fn(n, m, pp, s1, len(sigma1), s2, len(sigma2)))


def lb1(p, sigma1, sigma2, minht=False) -> int:
    """LB1 of the node (sigma1, sigma2); minht: with the heads and tails refinement."""
    return _bound(lib().orc_lb1_minht if minht else lib().orc_lb1, p, sigma1, sigma2)


def lb2(p, sigma1, sigma2) -> int:
    return _bound(lib().orc_lb2, p, sigma1, sigma2)


def pair_value(p, k, l, front_, back_, seq) -> int:
    n, m = _shape(p)
    P, pp = _i32(p)
    F, fp = _i32(front_)
    B, bp = _i32(back_)
    S, sp = _i32(list(seq) or [0])
    return int(lib().orc_pair_value(n, m, pp, k, l, fp, bp, sp, len(seq)))


def johnson_lag_order(x, y, g):
    X, xp = _i32(x)
    Y, yp = _i32(y)
    G, gp = _i32(g)
    O, op = _i32(np.zeros(len(X)))
    lib().orc_johnson_lag_order(len(X), xp, yp, gp, op)
    return O


def johnson(p):
    n, m = _shape(p)
    assert m == 2
    P, pp = _i32(p)
    O, op = _i32(np.zeros(n))
    c = int(lib().orc_johnson(n, pp, op))
    return c, O


def children_bounds(p, perm, d1, d2, kind=LB1 | LB2):
    """Bounds of all children of node [perm, d1, d2]: arrays [2, n] (dir, job), -1 if scheduled."""
    n, m = _shape(p)
    P, pp = _i32(p)
    Q, qp = _u8(perm)
    o1, op1 = _i32(np.zeros(2 * n))
    o2, op2 = _i32(np.zeros(2 * n))
    lib().orc_children_bounds(n, m, pp, kind, qp, int(d1), int(d2), op1, op2)
    return o1.reshape(2, n), o2.reshape(2, n)


def children_bounds_batch(p, perm, d1, d2, kind=LB1 | LB2, threads=1, pairs=None):
    """Bounds of both children sets of every node; pairs (indices in k < l order)
    restricts LB2 to those machine pairs (LB2 = max(LB1, their values)); the MINHT
    bit of kind refines LB1's empty heads and tails (LB2 = max(that LB1, pairs))."""
    n, m = _shape(p)
    count = len(d1)
    P, pp = _i32(p)
    Q, qp = _u8(perm)
    D1, dp1 = _u8(d1)
    D2, dp2 = _u8(d2)
    o1 = np.empty(count * 2 * n, dtype=np.int32)
    o2 = np.empty(count * 2 * n, dtype=np.int32)
    Sp, sp = _i32(pairs if pairs is not None else [0])
    lib().orc_children_bounds_batch_pairs(n, m, pp, kind, count, qp, dp1, dp2,
                                          o1.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          o2.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), threads,
                                          sp if pairs is not None else None,
                                          len(pairs) if pairs is not None else 0)
    return o1.reshape(count, 2, n), o2.reshape(count, 2, n)


def minmin(lbf, lbb, unscheduled, cap=INT32_MAX) -> int:
    n = len(lbf)
    F, fp = _i32(lbf)
    B, bp = _i32(lbb)
    un = np.zeros(n, dtype=np.uint8)
    un[list(unscheduled)] = 1
    U, up = _u8(un)
    return int(lib().orc_minmin(n, fp, bp, up, cap))


def branch_rule(lbf, lbb, unscheduled, rule, cap=INT32_MAX) -> int:
    """Direction (0 forward, 1 backward) chosen by branching rule `rule` (MINMIN, MINMIN_CAPPED,
    MINBRANCH or MINSUM); cap is the solve's initial incumbent."""
    n = len(lbf)
    F, fp = _i32(lbf)
    B, bp = _i32(lbb)
    un = np.zeros(n, dtype=np.uint8)
    un[list(unscheduled)] = 1
    U, up = _u8(un)
    return int(lib().orc_branch_rule(n, fp, bp, up, int(rule), int(cap)))


def bb_solve(p, bound=LB1, init_ub=INT32_MAX, node_limit=0, capped=False, pairs=None, branching=None,
             minht=False):
    """Sequential DFS branch-and-bound (LB2 over `pairs` when given).  `branching` is one of
    MINMIN, MINMIN_CAPPED, MINBRANCH, MINSUM (default: MinMin, capped when `capped`); minht
    refines LB1's empty heads and tails.
    Returns dict(outcome, cmax, perm, decomposed, bounded, leaves, pruned)."""
    bound = int(bound) | (MINHT if minht else 0)
    rule = (MINMIN_CAPPED if capped else MINMIN) if branching is None else int(branching)
    n, m = _shape(p)
    P, pp = _i32(p)
    best = np.zeros(1, dtype=np.int32)
    perm = np.full(n, -1, dtype=np.int32)
    cnt = np.zeros(4, dtype=np.int64)
    Sp, sp = _i32(pairs if pairs is not None else [0])
    out = lib().orc_bb_solve_pairs(n, m, pp, bound, rule, int(init_ub), int(node_limit),
                                   best.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   sp if pairs is not None else None, len(pairs) if pairs is not None else 0)
    return dict(outcome=int(out), cmax=int(best[0]), perm=perm, decomposed=int(cnt[0]),
                bounded=int(cnt[1]), leaves=int(cnt[2]), pruned=int(cnt[3]))


def brute_force(p):
    n, m = _shape(p)
    P, pp = _i32(p)
    O, op = _i32(np.zeros(n))
    c = int(lib().orc_brute_force(n, m, pp, op))
    return c, O


def neh(p):
    n, m = _shape(p)
    P, pp = _i32(p)
    O, op = _i32(np.zeros(n))
    c = int(lib().orc_neh(n, m, pp, op))
    return c, O


def factoradic_from_decimal(n, x):
    D, dp = _i32(np.zeros(n))
    lib().orc_factoradic_from_decimal(n, int(x), dp)
    return D


def factoradic_to_decimal(digits) -> int:
    D, dp = _i32(digits)
    return int(lib().orc_factoradic_to_decimal(len(D), dp))


def steal_midpoint(a, b) -> int:
    return int(lib().orc_steal_midpoint(int(a), int(b)))


def ivm_decode(jobs, dirs):
    level = len(jobs) - 1
    J, jp = _i32(jobs)
    Dd, dp = _i32(dirs)
    s1, s1p = _i32(np.zeros(len(jobs)))
    s2, s2p = _i32(np.zeros(len(jobs)))
    a = np.zeros(1, dtype=np.int32)
    b = np.zeros(1, dtype=np.int32)
    lib().orc_ivm_decode(level, jp, dp, s1p, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         s2p, b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return list(s1[:a[0]]), list(s2[:b[0]])
