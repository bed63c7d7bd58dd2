"""Seeded synthetic inputs for the PFSP branch-and-bound hot path.

This module holds only random-number generation and the shapes of the
workloads; it contains none of the method's arithmetic (no makespan, no bound,
no branching).  Both the CUDA path's tests/benchmarks and the CPU oracle's
tests draw their inputs from here, so the two sides see identical data.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written from its published definition.

Processing times follow the value distribution of the paper's benchmark
classes (Section 5: Taillard and VFR instances draw integer times uniformly
from [1, 99]); the instances themselves are synthetic, not Taillard's or VFR's.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: int, count: int) -> np.ndarray:
    """Return `count` consecutive SplitMix64 outputs starting from `state`.

    Output i is mix(state + (i + 1) * golden), where mix is the published
    finaliser (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31).
    """
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(state & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def instance_state(n: int, m: int, seed: int) -> int:
    """Starting state of the stream for an n x m instance with a given seed."""
    return (seed * 0x100000001B3 + (n << 40) + (m << 48)) & 0xFFFFFFFFFFFFFFFF


def make_instance(n: int, m: int, seed: int, lo: int = 1, hi: int = 99) -> np.ndarray:
    """Processing-time matrix p[j, k] (job-major, int32), uniform in [lo, hi].

    p[j, k] = lo + (x_{j*m+k} mod (hi - lo + 1)) with x the SplitMix64 stream.
    """
    x = splitmix64(instance_state(n, m, seed), n * m)
    span = np.uint64(hi - lo + 1)
    p = (x % span).astype(np.int64) + lo
    return p.astype(np.int32).reshape(n, m)


def batch_instance_shape(i: int) -> tuple[int, int]:
    """Shape (n, m) of instance i of the uneven multi-instance batch.

    h_i is the first SplitMix64 output of stream i; n = 12 + (h_i mod 9) and
    m is 5, 10 or 20 by (h_i >> 8) mod 3.
    """
    h = int(splitmix64(0xB47C4 + i * 0x1000193, 1)[0])
    n = 12 + (h % 9)
    m = (5, 10, 20)[(h >> 8) % 3]
    return n, m


def random_nodes(n: int, count: int, seed: int, dmax: int = 10, chunk: int = 1 << 20):
    """Random partial schedules for the bounding microbenchmark.

    Each node is a uniformly random permutation of the n jobs (ordering by
    SplitMix64 keys, ties impossible in practice and broken by job id) and two
    depths d1, d2 drawn independently and uniformly from {0, ..., dmax}, with
    d1 + d2 <= n enforced by clipping d2.  The first d1 entries of the
    permutation are the prefix schedule, the last d2 the suffix schedule, so
    the two job sets are disjoint by construction.

    Returns (perm uint8[count, n], d1 uint8[count], d2 uint8[count]).
    """
    perm = np.empty((count, n), dtype=np.uint8)
    d1 = np.empty(count, dtype=np.uint8)
    d2 = np.empty(count, dtype=np.uint8)
    base = (seed * 0x2545F4914F6CDD1D + n) & 0xFFFFFFFFFFFFFFFF
    for start in range(0, count, chunk):
        c = min(chunk, count - start)
        keys = splitmix64(base + start * (n + 2) * 0x9E3779B97F4A7C15, c * (n + 2))
        keys = keys.reshape(c, n + 2)
        perm[start:start + c] = np.argsort(keys[:, :n], axis=1, kind="stable").astype(np.uint8)
        a = (keys[:, n] % np.uint64(dmax + 1)).astype(np.int64)
        b = (keys[:, n + 1] % np.uint64(dmax + 1)).astype(np.int64)
        b = np.minimum(b, n - a)
        d1[start:start + c] = a
        d2[start:start + c] = b
    return perm, d1, d2


def all_nodes_small(n: int):
    """Every partial schedule (perm, d1, d2) of an n-job problem, for tiny n.

    Enumerates each ordered prefix sigma1, each ordered suffix sigma2 on the
    remaining jobs, and lists the unscheduled jobs in ascending order.  Used for
    exhaustive checks at n <= 5.
    """
    import itertools

    perms, d1s, d2s = [], [], []
    jobs = list(range(n))
    for a in range(n + 1):
        for s1 in itertools.permutations(jobs, a):
            rest = [j for j in jobs if j not in s1]
            for b in range(len(rest) + 1):
                for s2 in itertools.permutations(rest, b):
                    mid = [j for j in rest if j not in s2]
                    perms.append(list(s1) + mid + list(s2))
                    d1s.append(a)
                    d2s.append(b)
    return (np.array(perms, dtype=np.uint8).reshape(-1, n),
            np.array(d1s, dtype=np.uint8), np.array(d2s, dtype=np.uint8))
