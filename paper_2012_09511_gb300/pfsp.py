"""Thin Python binding of the C ABI in include/pfsp.h (ctypes; marshalling only).

Every function here has the name of the C entry point it calls and does no
computation of its own: all bounding and searching runs in the CUDA library
libpfsp_gb300.so.  If that library is missing, importing this module fails
loudly; there is no CPU fallback.

Host-pointer entry points take numpy arrays; the _dev entry points take device
addresses (e.g. torch.Tensor.data_ptr()) and a stream handle
(torch.cuda.Stream.cuda_stream), both as Python ints.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpfsp_gb300.so")

PFSP_OK = 0
PFSP_ERR_INVALID = -1
PFSP_ERR_OOM = -2
PFSP_ERR_CUDA = -3
PFSP_ERR_UNSUPPORTED = -4
PFSP_ERR_TIMEOUT = -5
PFSP_OPTIMAL = 0
PFSP_PROVEN_NO_BETTER = 1
PFSP_LIMIT_NODES = 2
PFSP_LIMIT_TIME = 3
PFSP_LB1 = 1
PFSP_LB2 = 2
PFSP_MINHT = 4
PFSP_MINMIN = 0
PFSP_MINMIN_CAPPED = 1
PFSP_MINBRANCH = 2
PFSP_MINSUM = 3
INT32_MAX = 2**31 - 1


class PfspError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pfsp error %d: %s" % (code, msg))
        self.code = code


class pfsp_stats_t(ctypes.Structure):
    _fields_ = [("decomposed", ctypes.c_uint64), ("bounded_children", ctypes.c_uint64),
                ("leaves", ctypes.c_uint64), ("pruned", ctypes.c_uint64), ("steals", ctypes.c_uint64),
                ("iterations", ctypes.c_uint64), ("seconds", ctypes.c_double),
                ("kernel_seconds", ctypes.c_double), ("final_ub", ctypes.c_int32),
                ("explorers", ctypes.c_int32), ("phase_cycles", ctypes.c_uint64 * 8), ("lb2_slots", ctypes.c_uint64),
                ("heuristic_improvements", ctypes.c_uint64), ("promoted", ctypes.c_uint64),
                ("heuristic_cmax", ctypes.c_int32), ("snapshots", ctypes.c_int32)]

    PHASES = ("service", "select", "decode", "lb1", "lb2", "branch", "init", "idle")

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "phase_cycles"}
        d["phase_cycles"] = dict(zip(self.PHASES, [int(x) for x in self.phase_cycles]))
        return d


PFSP_LEARN_CHILD_ORDER = 1
PFSP_LEARN_PAIR_ORDER = 2
PFSP_EARLY_EXIT = 4
PFSP_EARLY_EXIT_SLOTS = 8
PFSP_EARLY_EXIT_CHILDREN = 16


class pfsp_options(ctypes.Structure):
    _fields_ = [("init_ub", ctypes.c_int32), ("node_limit", ctypes.c_int64), ("time_limit_s", ctypes.c_double),
                ("bound", ctypes.c_int), ("branching", ctypes.c_int), ("warps_per_sm", ctypes.c_int),
                ("check_every", ctypes.c_int), ("min_steal", ctypes.c_double), ("mlp", ctypes.c_void_p),
                ("learned", ctypes.c_int), ("learn_depth", ctypes.c_int), ("phase_timers", ctypes.c_int),
                ("heuristic_threads", ctypes.c_int), ("heuristic_seed", ctypes.c_int), ("lb1_minht", ctypes.c_int),
                ("heuristic_kind", ctypes.c_int), ("slot_warps", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


if not os.path.exists(LIB_PATH):
    raise ImportError("libpfsp_gb300.so is not built (run __graft_entry__.build()); "
                      "the library has no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_lib.pfsp_last_error.restype = ctypes.c_char_p
_lib.pfsp_last_error.argtypes = []
_lib.pfsp_load_instance.restype = ctypes.c_int
_lib.pfsp_load_instance.argtypes = [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_lib.pfsp_free_instance.restype = None
_lib.pfsp_free_instance.argtypes = [_vp]
_lib.pfsp_bound_batch.restype = ctypes.c_int
_lib.pfsp_bound_batch.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
_lib.pfsp_bound_batch_dev.restype = ctypes.c_int
_lib.pfsp_bound_batch_dev.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.pfsp_bound_reduce.restype = ctypes.c_int
_lib.pfsp_bound_reduce.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32, _vp]
_lib.pfsp_bound_reduce_dev.restype = ctypes.c_int
_lib.pfsp_bound_reduce_dev.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp]
_lib.pfsp_default_options.restype = None
_lib.pfsp_default_options.argtypes = [ctypes.POINTER(pfsp_options)]
_lib.pfsp_solve.restype = ctypes.c_int
_lib.pfsp_solve.argtypes = [_vp, ctypes.POINTER(pfsp_options), ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int)]
_lib.pfsp_solve_noalloc.restype = ctypes.c_int
_lib.pfsp_solve_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(pfsp_options),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(pfsp_stats_t)]
_lib.pfsp_solve_batch.restype = ctypes.c_int
_lib.pfsp_solve_batch.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(pfsp_options), _vp,
                                  _vp, _vp, _vp, ctypes.POINTER(pfsp_stats_t)]
_lib.pfsp_iterated_greedy.restype = ctypes.c_int
_lib.pfsp_iterated_greedy.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int64, ctypes.c_uint64,
                                      _vp, ctypes.POINTER(ctypes.c_int32)]
_lib.pfsp_beam_search.restype = ctypes.c_int
_lib.pfsp_beam_search.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int,
                                  _vp, ctypes.POINTER(ctypes.c_int32)]
_lib.pfsp_autotune_batch.restype = ctypes.c_int
_lib.pfsp_autotune_batch.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(pfsp_options),
                                     ctypes.c_int, ctypes.POINTER(pfsp_options)]
_fp = ctypes.POINTER(ctypes.c_float)
_lib.pfsp_mlp_create.restype = ctypes.c_int
_lib.pfsp_mlp_create.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(_vp)]
_lib.pfsp_mlp_free.restype = None
_lib.pfsp_mlp_free.argtypes = [_vp]
_lib.pfsp_mlp_shape.restype = ctypes.c_int
_lib.pfsp_mlp_shape.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int)] * 4 + [ctypes.POINTER(ctypes.c_int64)]
_lib.pfsp_mlp_get_params.restype = ctypes.c_int
_lib.pfsp_mlp_get_params.argtypes = [_vp, _vp]
_lib.pfsp_mlp_set_params.restype = ctypes.c_int
_lib.pfsp_mlp_set_params.argtypes = [_vp, _vp]
_lib.pfsp_mlp_forward.restype = ctypes.c_int
_lib.pfsp_mlp_forward.argtypes = [_vp, ctypes.c_int64, _vp, _vp]
_lib.pfsp_mlp_loss_grad.restype = ctypes.c_int
_lib.pfsp_mlp_loss_grad.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
_lib.pfsp_mlp_train.restype = ctypes.c_int
_lib.pfsp_mlp_train.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                ctypes.c_uint64, _vp]
_lib.pfsp_solve_trace.restype = ctypes.c_int
_lib.pfsp_solve_trace.argtypes = [_vp, ctypes.POINTER(pfsp_options), ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp,
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int)]
_lib.pfsp_mlp_rows.restype = ctypes.c_int
_lib.pfsp_mlp_rows.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.pfsp_stats.restype = ctypes.c_int
_lib.pfsp_stats.argtypes = [_vp, ctypes.POINTER(pfsp_stats_t)]
_lib.pfsp_solve_resumable.restype = ctypes.c_int
_lib.pfsp_solve_resumable.argtypes = [_vp, ctypes.POINTER(pfsp_options), _vp, ctypes.c_int64, ctypes.POINTER(_vp),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int)]
_lib.pfsp_free_checkpoint.restype = None
_lib.pfsp_free_checkpoint.argtypes = [_vp]
_lib.pfsp_set_pair_order.restype = ctypes.c_int
_lib.pfsp_set_pair_order.argtypes = [_vp, _vp]
_lib.pfsp_set_steal_wait_limit.restype = ctypes.c_int
_lib.pfsp_set_steal_wait_limit.argtypes = [ctypes.c_int]
_lib.pfsp_learn_lb2_pairs.restype = ctypes.c_int
_lib.pfsp_learn_lb2_pairs.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int, _vp]
_lib.pfsp_set_lb2_pairs.restype = ctypes.c_int
_lib.pfsp_set_lb2_pairs.argtypes = [_vp, _vp, ctypes.c_int]
_lib.pfsp_get_pair_order.restype = ctypes.c_int
_lib.pfsp_get_pair_order.argtypes = [_vp, _vp]
_lib.pfsp_mlp_pair_scores.restype = ctypes.c_int
_lib.pfsp_mlp_pair_scores.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
_lib.pfsp_learn_pair_order.restype = ctypes.c_int
_lib.pfsp_learn_pair_order.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp]


def lib():
    """The loaded ctypes library (for symbol checks and extensions)."""
    return _lib


def pfsp_last_error() -> str:
    return _lib.pfsp_last_error().decode()


def _check(rc):
    if rc < 0:
        raise PfspError(rc, pfsp_last_error())
    return rc


def _ptr(a):
    return a.ctypes.data_as(_vp) if a is not None else None


class Instance:
    """Owner of a pfsp_instance handle; frees it on close or garbage collection."""

    def __init__(self, handle, n, m):
        self.handle = handle
        self.n = n
        self.m = m

    def close(self):
        if self.handle:
            _lib.pfsp_free_instance(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pfsp_load_instance(p) -> Instance:
    """p: int array [n, m] (job-major)."""
    p = np.ascontiguousarray(p, dtype=np.int32)
    n, m = p.shape
    h = _vp()
    _check(_lib.pfsp_load_instance(n, m, _ptr(p), ctypes.byref(h)))
    return Instance(h, n, m)


def pfsp_free_instance(inst: Instance) -> None:
    inst.close()


def pfsp_bound_batch(inst: Instance, kind, perm, d1, d2, lb1_out=None, lb2_out=None):
    """Host buffers: perm uint8 [N, n], d1/d2 uint8 [N].  Returns (lb1, lb2), each int32
    [N, 2, n] or None when not requested."""
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    d1 = np.ascontiguousarray(d1, dtype=np.uint8)
    d2 = np.ascontiguousarray(d2, dtype=np.uint8)
    N = len(d1)
    n = inst.n
    if kind & PFSP_LB1 and lb1_out is None:
        lb1_out = np.empty((N, 2, n), dtype=np.int32)
    if kind & PFSP_LB2 and lb2_out is None:
        lb2_out = np.empty((N, 2, n), dtype=np.int32)
    _check(_lib.pfsp_bound_batch(inst.handle, kind, N, _ptr(perm), _ptr(d1), _ptr(d2),
                                 _ptr(lb1_out) if kind & PFSP_LB1 else None,
                                 _ptr(lb2_out) if kind & PFSP_LB2 else None))
    return (lb1_out if kind & PFSP_LB1 else None), (lb2_out if kind & PFSP_LB2 else None)


def pfsp_bound_batch_dev(inst: Instance, kind, num_nodes, perm, d1, d2, lb1_out, lb2_out, stream=0):
    """Device addresses as ints (0 = NULL); enqueues on `stream` and returns."""
    _check(_lib.pfsp_bound_batch_dev(inst.handle, kind, int(num_nodes), perm or None, d1 or None,
                                     d2 or None, lb1_out or None, lb2_out or None, stream or None))


# pfsp_node_summary: per parent and direction (0 forward, 1 backward)
SUMMARY_DTYPE = np.dtype([("min", "<i4", (2,)), ("count", "<i4", (2,)), ("sum", "<i8", (2,)),
                          ("keep", "<u8", (2,))])
assert SUMMARY_DTYPE.itemsize == 48


def pfsp_bound_reduce(inst: Instance, kind, perm, d1, d2, ub, out=None) -> np.ndarray:
    """Reduce mode on host buffers: one SUMMARY_DTYPE record per node (survivors below ub)."""
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    d1 = np.ascontiguousarray(d1, dtype=np.uint8)
    d2 = np.ascontiguousarray(d2, dtype=np.uint8)
    N = len(d1)
    if out is None:
        out = np.empty(N, dtype=SUMMARY_DTYPE)
    _check(_lib.pfsp_bound_reduce(inst.handle, kind, N, _ptr(perm), _ptr(d1), _ptr(d2), int(ub), _ptr(out)))
    return out


def pfsp_bound_reduce_dev(inst: Instance, kind, num_nodes, perm, d1, d2, ub, out, stream=0):
    """Reduce mode on device addresses (ints); enqueues on `stream` and returns."""
    _check(_lib.pfsp_bound_reduce_dev(inst.handle, kind, int(num_nodes), perm or None, d1 or None, d2 or None,
                                      int(ub), out or None, stream or None))


def pfsp_stats(inst: Instance) -> dict:
    s = pfsp_stats_t()
    _check(_lib.pfsp_stats(inst.handle, ctypes.byref(s)))
    return s.as_dict()


def pfsp_default_options(**fields) -> pfsp_options:
    """Defaults of the library, then the given fields (names as in the C struct;
    `mlp` may be an Mlp object)."""
    o = pfsp_options()
    _lib.pfsp_default_options(ctypes.byref(o))
    for k, v in fields.items():
        if k == "mlp" and v is not None and not isinstance(v, int):
            o._mlp_owner = v  # keep the network alive with the options
            v = v.handle.value if hasattr(v.handle, "value") else v.handle
        setattr(o, k, v)
    return o


def pfsp_solve(inst: Instance, opts: pfsp_options = None, **fields) -> dict:
    """Solve; returns dict(cmax, perm, outcome, **stats)."""
    if opts is None:
        opts = pfsp_default_options(**fields)
    best = ctypes.c_int32()
    out = ctypes.c_int()
    perm = (ctypes.c_int32 * inst.n)(*([-1] * inst.n))
    _check(_lib.pfsp_solve(inst.handle, ctypes.byref(opts), ctypes.byref(best), perm, ctypes.byref(out)))
    r = dict(cmax=best.value, perm=np.array(perm[:], dtype=np.int32), outcome=out.value)
    r.update(pfsp_stats(inst))
    return r


def pfsp_iterated_greedy(p, iterations, seed=0, start=None):
    """Host iterated greedy on p ([n, m] job-major) from `start` (None: NEH).
    Returns (cmax, perm)."""
    p = np.ascontiguousarray(p, dtype=np.int32)
    n, m = p.shape
    s = None if start is None else np.ascontiguousarray(start, dtype=np.int32)
    perm = np.full(n, -1, dtype=np.int32)
    c = ctypes.c_int32()
    _check(_lib.pfsp_iterated_greedy(_ptr(p), n, m, _ptr(s), int(iterations), int(seed), _ptr(perm), ctypes.byref(c)))
    return c.value, perm


def pfsp_beam_search(p, width, prefix=(), suffix=()):
    """Host beam search on p ([n, m] job-major) below the node (prefix, suffix).
    Returns (cmax, perm)."""
    p = np.ascontiguousarray(p, dtype=np.int32)
    n, m = p.shape
    a = np.ascontiguousarray(list(prefix) or [0], dtype=np.int32)
    b = np.ascontiguousarray(list(suffix) or [0], dtype=np.int32)
    perm = np.full(n, -1, dtype=np.int32)
    c = ctypes.c_int32()
    _check(_lib.pfsp_beam_search(_ptr(p), n, m, _ptr(a), len(prefix), _ptr(b), len(suffix), int(width), _ptr(perm),
                                 ctypes.byref(c)))
    return c.value, perm


def pfsp_solve_noalloc(p, opts: pfsp_options = None, **fields) -> dict:
    """pfsp_solve without device allocations (static scratch); p is [n, m] job-major."""
    p = np.ascontiguousarray(p, dtype=np.int32)
    n, m = p.shape
    if opts is None:
        opts = pfsp_default_options(**fields)
    best = ctypes.c_int32()
    out = ctypes.c_int()
    perm = (ctypes.c_int32 * n)(*([-1] * n))
    st = pfsp_stats_t()
    _check(_lib.pfsp_solve_noalloc(n, m, _ptr(p), ctypes.byref(opts), ctypes.byref(best), perm,
                                   ctypes.byref(out), ctypes.byref(st)))
    r = dict(cmax=best.value, perm=np.array(perm[:], dtype=np.int32), outcome=out.value)
    r.update(st.as_dict())
    return r


def _handles(insts):
    arr = (_vp * len(insts))(*[i.handle for i in insts])
    return arr


def pfsp_solve_batch(insts, opts: pfsp_options = None, init_ubs=None, **fields) -> dict:
    """Solve a list of Instances in one launch.  Returns dict(cmax [count], perms [count, 64],
    outcomes [count], stats)."""
    if opts is None:
        opts = pfsp_default_options(**fields)
    k = len(insts)
    cm = np.zeros(k, dtype=np.int32)
    out = np.zeros(k, dtype=np.int32)
    perms = np.zeros((k, 64), dtype=np.int32)
    ubs = None if init_ubs is None else np.ascontiguousarray(init_ubs, dtype=np.int32)
    st = pfsp_stats_t()
    _check(_lib.pfsp_solve_batch(_handles(insts), k, ctypes.byref(opts), _ptr(ubs), _ptr(cm), _ptr(perms),
                                 _ptr(out), ctypes.byref(st)))
    return dict(cmax=cm, perms=perms, outcomes=out, stats=st.as_dict())


def pfsp_autotune_batch(insts, base: pfsp_options = None, sample=0) -> pfsp_options:
    if base is None:
        base = pfsp_default_options()
    best = pfsp_options()
    _check(_lib.pfsp_autotune_batch(_handles(insts), len(insts), ctypes.byref(base), int(sample),
                                    ctypes.byref(best)))
    return best


class Mlp:
    """Owner of a pfsp_mlp handle (the ordering network)."""

    def __init__(self, handle):
        self.handle = handle
        d0, h, o, p = (ctypes.c_int() for _ in range(4))
        n = ctypes.c_int64()
        _check(_lib.pfsp_mlp_shape(handle, ctypes.byref(d0), ctypes.byref(h), ctypes.byref(o), ctypes.byref(p),
                                   ctypes.byref(n)))
        self.D0, self.H, self.O, self.P, self.n_params = d0.value, h.value, o.value, p.value, n.value

    def close(self):
        if self.handle:
            _lib.pfsp_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def split(self, flat):
        """[W1, b1, W2, b2, W3, b3] views of a flat parameter vector."""
        D0, H, O = self.D0, self.H, self.O
        sizes = [D0 * H, H, H * H, H, H * O, O]
        shapes = [(D0, H), (H,), (H, H), (H,), (H, O), (O,)]
        out, o = [], 0
        for sz, sh in zip(sizes, shapes):
            out.append(flat[o:o + sz].reshape(sh))
            o += sz
        return out


def pfsp_mlp_create(m, seed=0) -> Mlp:
    h = _vp()
    _check(_lib.pfsp_mlp_create(int(m), int(seed), ctypes.byref(h)))
    return Mlp(h)


def pfsp_mlp_free(mlp: Mlp) -> None:
    mlp.close()


def pfsp_mlp_get_params(mlp: Mlp) -> np.ndarray:
    out = np.empty(mlp.n_params, dtype=np.float32)
    _check(_lib.pfsp_mlp_get_params(mlp.handle, _ptr(out)))
    return out


def pfsp_mlp_set_params(mlp: Mlp, flat) -> None:
    flat = np.ascontiguousarray(flat, dtype=np.float32)
    assert flat.size == mlp.n_params
    _check(_lib.pfsp_mlp_set_params(mlp.handle, _ptr(flat)))


def pfsp_mlp_forward(mlp: Mlp, X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.empty((X.shape[0], mlp.O), dtype=np.float32)
    _check(_lib.pfsp_mlp_forward(mlp.handle, X.shape[0], _ptr(X), _ptr(Y)))
    return Y


def pfsp_mlp_loss_grad(mlp: Mlp, X, T, M):
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    M = np.ascontiguousarray(M, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.empty(mlp.n_params, dtype=np.float32)
    _check(_lib.pfsp_mlp_loss_grad(mlp.handle, X.shape[0], _ptr(X), _ptr(T), _ptr(M), _ptr(loss), _ptr(grad)))
    return float(loss[0]), grad


def pfsp_mlp_train(mlp: Mlp, X, T, M, epochs=5, batch=4096, lr=1e-3, seed=0) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    M = np.ascontiguousarray(M, dtype=np.float32)
    losses = np.zeros(epochs, dtype=np.float32)
    _check(_lib.pfsp_mlp_train(mlp.handle, X.shape[0], _ptr(X), _ptr(T), _ptr(M), int(epochs), int(batch),
                               float(lr), int(seed), _ptr(losses)))
    return losses


def pfsp_solve_trace(inst: Instance, capacity, stride=1, opts: pfsp_options = None, **fields):
    """Solve while recording every stride-th decomposition: returns (perm [k, n], d1 [k], d2 [k], result)."""
    if opts is None:
        opts = pfsp_default_options(**fields)
    n = inst.n
    perm = np.zeros((max(capacity, 1), n), dtype=np.uint8)
    d1 = np.zeros(max(capacity, 1), dtype=np.uint8)
    d2 = np.zeros(max(capacity, 1), dtype=np.uint8)
    cnt = ctypes.c_int64()
    best = ctypes.c_int32()
    out = ctypes.c_int()
    _check(_lib.pfsp_solve_trace(inst.handle, ctypes.byref(opts), int(capacity), int(stride), _ptr(perm), _ptr(d1),
                                 _ptr(d2), ctypes.byref(cnt), ctypes.byref(best), ctypes.byref(out)))
    k = cnt.value
    r = dict(cmax=best.value, outcome=out.value)
    r.update(pfsp_stats(inst))
    return perm[:k], d1[:k], d2[:k], r


def pfsp_mlp_rows(inst: Instance, mlp: Mlp, perm, d1, d2):
    """Training rows (X, T, M) of the nodes: (1 + 2n) rows per node."""
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    d1 = np.ascontiguousarray(d1, dtype=np.uint8)
    d2 = np.ascontiguousarray(d2, dtype=np.uint8)
    k = len(d1)
    rows = k * (1 + 2 * inst.n)
    X = np.empty((rows, mlp.D0), dtype=np.float32)
    T = np.empty((rows, mlp.O), dtype=np.float32)
    M = np.empty((rows, mlp.O), dtype=np.float32)
    _check(_lib.pfsp_mlp_rows(inst.handle, mlp.handle, k, _ptr(perm), _ptr(d1), _ptr(d2), _ptr(X), _ptr(T),
                              _ptr(M)))
    return X, T, M


def pfsp_set_steal_wait_limit(polls: int = 0) -> None:
    """Test hook: polls of a thief's answer wait in pfsp_solve (0 = the default)."""
    _check(_lib.pfsp_set_steal_wait_limit(int(polls)))


def pfsp_set_pair_order(inst: Instance, order=None) -> None:
    """Sweep order of the machine pairs (indices k < l lexicographic); None = index order."""
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    _check(_lib.pfsp_set_pair_order(inst.handle, _ptr(o)))


def pfsp_set_lb2_pairs(inst: Instance, pairs=None) -> None:
    """LB2 over the listed machine pairs only (indices in k < l order); None = all pairs."""
    q = None if pairs is None else np.ascontiguousarray(pairs, dtype=np.int32)
    _check(_lib.pfsp_set_lb2_pairs(inst.handle, _ptr(q), 0 if q is None else len(q)))


def pfsp_get_pair_order(inst: Instance) -> np.ndarray:
    """The pairs LB2 uses, in sweep order."""
    out = np.empty(inst.m * (inst.m - 1) // 2, dtype=np.int32)
    _check(_lib.pfsp_get_pair_order(inst.handle, _ptr(out)))
    return out[out >= 0]


def pfsp_mlp_pair_scores(inst: Instance, mlp: Mlp, perm, d1, d2) -> np.ndarray:
    """Mean network probability per pair over the nodes (pair index order)."""
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    d1 = np.ascontiguousarray(d1, dtype=np.uint8)
    d2 = np.ascontiguousarray(d2, dtype=np.uint8)
    out = np.empty(max(1, inst.m * (inst.m - 1) // 2), dtype=np.float32)
    _check(_lib.pfsp_mlp_pair_scores(inst.handle, mlp.handle, len(d1), _ptr(perm), _ptr(d1), _ptr(d2), _ptr(out)))
    return out[:inst.m * (inst.m - 1) // 2]


def pfsp_learn_pair_order(inst: Instance, mlp: Mlp, perm, d1, d2) -> np.ndarray:
    """Rank the pairs by the network's scores over the nodes and apply that order; returns it."""
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    d1 = np.ascontiguousarray(d1, dtype=np.uint8)
    d2 = np.ascontiguousarray(d2, dtype=np.uint8)
    out = np.empty(max(1, inst.m * (inst.m - 1) // 2), dtype=np.int32)
    _check(_lib.pfsp_learn_pair_order(inst.handle, mlp.handle, len(d1), _ptr(perm), _ptr(d1), _ptr(d2), _ptr(out)))
    return out[:inst.m * (inst.m - 1) // 2]


def pfsp_solve_resumable(inst: Instance, resume: bytes = None, opts: pfsp_options = None, **fields) -> dict:
    """One segment of a resumable solve; returns dict(cmax, perm, outcome, checkpoint, **stats), where
    checkpoint is the bytes to resume from (None once the search has finished)."""
    if opts is None:
        opts = pfsp_default_options(**fields)
    best = ctypes.c_int32()
    out = ctypes.c_int()
    perm = (ctypes.c_int32 * inst.n)(*([-1] * inst.n))
    ck = _vp()
    nb = ctypes.c_int64()
    rb = None if resume is None else ctypes.create_string_buffer(bytes(resume), len(resume))
    _check(_lib.pfsp_solve_resumable(inst.handle, ctypes.byref(opts), rb, len(resume) if resume else 0,
                                     ctypes.byref(ck), ctypes.byref(nb), ctypes.byref(best), perm, ctypes.byref(out)))
    data = None
    if ck.value:
        data = ctypes.string_at(ck.value, nb.value)
        _lib.pfsp_free_checkpoint(ck)
    r = dict(cmax=best.value, perm=np.array(perm[:], dtype=np.int32), outcome=out.value, checkpoint=data)
    r.update(pfsp_stats(inst))
    return r


def pfsp_learn_lb2_pairs(inst: Instance, mlp: Mlp, keep=32, perm=None, d1=None, d2=None) -> np.ndarray:
    """LB2 over the `keep` pairs the network scores highest (sample: the given nodes, or the
    root's children); returns the pairs kept, best first."""
    P = inst.m * (inst.m - 1) // 2
    out = np.empty(max(1, min(keep, P)), dtype=np.int32)
    if perm is None:
        _check(_lib.pfsp_learn_lb2_pairs(inst.handle, mlp.handle, 0, None, None, None, int(keep), _ptr(out)))
    else:
        perm = np.ascontiguousarray(perm, dtype=np.uint8)
        d1 = np.ascontiguousarray(d1, dtype=np.uint8)
        d2 = np.ascontiguousarray(d2, dtype=np.uint8)
        _check(_lib.pfsp_learn_lb2_pairs(inst.handle, mlp.handle, len(d1), _ptr(perm), _ptr(d1), _ptr(d2), int(keep),
                                         _ptr(out)))
    return out[:min(keep, P)]
