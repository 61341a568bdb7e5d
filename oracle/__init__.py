"""Plain serial CPU oracle for the flow-shop branch-and-bound bounding path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_1206_4973_gb300``)
and never imports it; the two meet only through the seeded inputs of
``paper_1206_4973_gb300.inputs``, which hold none of the method's arithmetic.

The arithmetic lives in ``fsp_oracle.c`` (plain C, int32, serial), compiled
with gcc into ``oracle/_build/libfsp_oracle.so`` by :func:`build`.  Each
function below cites the part of the paper it follows; the bound itself is
the two-machine Johnson bound with time lags whose O(m^2 n log n) cost
Sec. V-D states (the paper prints no formula), together with the one-machine
bounds.  Pins: see the header of ``fsp_oracle.c``.  Parity unpinned: the exact
node interleaving of a pool > 1 search after the incumbent improves.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfsp_oracle.so")
_lock = threading.Lock()
_lib = None

OK, INCOMPLETE, ERR_ARG, ERR_OOM = 0, 1, -1, -3
INF = 2**31 - 1
STATS = ("bounded", "branched", "pruned", "leaves", "iterations", "incumbent_updates")


def build(force: bool = False) -> str:
    """Compile fsp_oracle.c with gcc (portable flags: same results on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fno-strict-aliasing", "-fopenmp",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i64p = ctypes.POINTER(ctypes.c_int64)
            c_int, c_i32, c_i64 = ctypes.c_int, ctypes.c_int32, ctypes.c_int64
            sig = {
                "orc_num_pairs": (c_int, [c_int]),
                "orc_release_times": (None, [c_int, c_int, i32p, u8p, c_int, i32p]),
                "orc_makespan": (c_i32, [c_int, c_int, i32p, u8p, c_int]),
                "orc_check_node": (c_int, [c_int, u8p, c_int]),
                "orc_bound_pool": (c_int, [c_int, c_int, i32p, u8p, c_i64, c_int, c_int, i32p]),
                "orc_bound_pool_threads": (c_int, [c_int, c_int, i32p, u8p, c_i64, c_int, c_int, i32p, c_int]),
                "orc_bound_pool2": (c_int, [c_int, c_int, i32p, u8p, c_i64, c_int, i32p]),
                "orc_lb2_parts": (c_int, [c_int, c_int, i32p, u8p, c_int, c_int, i32p, i32p, i32p, i32p]),
                "orc_solve_bidir": (c_int, [c_int, c_int, i32p, c_i32, c_i64, c_i64, c_i64, i32p, u8p, i64p,
                                            i64p, c_i64]),
                "orc_lb_parts": (c_int, [c_int, c_int, i32p, u8p, c_int, c_int, i32p, i32p, i32p]),
                "orc_tables_dump": (c_int, [c_int, c_int, i32p, i32p, i32p, u8p]),
                "orc_bruteforce": (c_i32, [c_int, c_int, i32p, u8p]),
                "orc_neh": (c_i32, [c_int, c_int, i32p, u8p]),
                "orc_solve": (c_int, [c_int, c_int, i32p, c_i32, c_i64, c_i64, i64p, c_i64,
                                      u8p, c_i64, c_int, c_i64,
                                      i32p, u8p, i64p, i64p, c_i64, u8p, c_i64, i64p, c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _inst(p):
    p = np.ascontiguousarray(p, dtype=np.int32)
    if p.ndim != 2:
        raise ValueError("p must be n x m (job-major)")
    return p, p.shape[0], p.shape[1]


def num_pairs(m: int) -> int:
    return m * (m - 1) // 2


def pairs(m: int):
    """Machine pairs (k, l), k < l, in the oracle's numbering (k-major)."""
    return [(k, l) for k in range(m) for l in range(k + 1, m)]


def release_times(p, perm, d: int) -> np.ndarray:
    """Sec. II-B: machine release times after scheduling perm[0..d)."""
    p, n, m = _inst(p)
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    out = np.zeros(m, dtype=np.int32)
    _load().orc_release_times(n, m, _p(p, ctypes.c_int32), _p(perm, ctypes.c_uint8), int(d),
                              _p(out, ctypes.c_int32))
    return out


def makespan(p, perm) -> int:
    """Sec. II-B: completion time of the last job on the last machine."""
    p, n, m = _inst(p)
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    return int(_load().orc_makespan(n, m, _p(p, ctypes.c_int32), _p(perm, ctypes.c_uint8), len(perm)))


def tables(p):
    """Tails q[n,m], lags lag[P,n] and Johnson orders order[P,n] (pairs k-major)."""
    p, n, m = _inst(p)
    P = num_pairs(m)
    q = np.zeros((n, m), np.int32)
    lag = np.zeros((P, n), np.int32)
    order = np.zeros((P, n), np.uint8)
    rc = _load().orc_tables_dump(n, m, _p(p, ctypes.c_int32), _p(q, ctypes.c_int32),
                                 _p(lag, ctypes.c_int32), _p(order, ctypes.c_uint8))
    if rc != OK:
        raise ValueError("invalid instance")
    return q, lag, order


def lb_parts(p, perm, d: int, bound: int = 0):
    """The node bound and its parts: (LB, LB1, [LB_kl per pair]).  bound 1: the
    release times strengthened by the smallest head (fsp_oracle.c, orc_lb)."""
    p, n, m = _inst(p)
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    lb = ctypes.c_int32(0)
    lb1 = ctypes.c_int32(0)
    pv = np.zeros(max(num_pairs(m), 1), np.int32)
    rc = _load().orc_lb_parts(n, m, _p(p, ctypes.c_int32), _p(perm, ctypes.c_uint8), int(d), int(bound),
                              ctypes.byref(lb), ctypes.byref(lb1), _p(pv, ctypes.c_int32))
    if rc != OK:
        raise ValueError("invalid node")
    return int(lb.value), int(lb1.value), pv[: num_pairs(m)].copy()


def lb(p, perm, d: int, bound: int = 0) -> int:
    return lb_parts(p, perm, d, bound)[0]


def bound_pool(p, nodes, bound: int = 0) -> np.ndarray:
    """Bound every record of nodes (uint8 [count, stride]: perm[n], depth at byte n)."""
    p, n, m = _inst(p)
    nodes = np.ascontiguousarray(nodes, dtype=np.uint8)
    count, stride = nodes.shape
    out = np.zeros(count, np.int32)
    rc = _load().orc_bound_pool(n, m, _p(p, ctypes.c_int32), _p(nodes, ctypes.c_uint8), count,
                                stride, int(bound), _p(out, ctypes.c_int32))
    if rc != OK:
        raise ValueError(f"orc_bound_pool failed ({rc})")
    return out


def bound_pool_threads(p, nodes, threads: int = 0, bound: int = 0):
    """bound_pool with the nodes split over host threads (0 = all cores): the
    same per-node bound.  Returns (bounds, threads used)."""
    p, n, m = _inst(p)
    nodes = np.ascontiguousarray(nodes, dtype=np.uint8)
    count, stride = nodes.shape
    out = np.zeros(count, np.int32)
    rc = _load().orc_bound_pool_threads(n, m, _p(p, ctypes.c_int32), _p(nodes, ctypes.c_uint8), count,
                                        stride, int(bound), _p(out, ctypes.c_int32), int(threads))
    if rc < 1:
        raise ValueError(f"orc_bound_pool_threads failed ({rc})")
    return out, int(rc)


def bruteforce(p):
    """Optimum over all n! permutations and the lexicographically first optimal one."""
    p, n, m = _inst(p)
    perm = np.zeros(n, np.uint8)
    c = _load().orc_bruteforce(n, m, _p(p, ctypes.c_int32), _p(perm, ctypes.c_uint8))
    return int(c), perm


def neh(p):
    """NEH insertion heuristic: (makespan, permutation)."""
    p, n, m = _inst(p)
    perm = np.zeros(n, np.uint8)
    c = _load().orc_neh(n, m, _p(p, ctypes.c_int32), _p(perm, ctypes.c_uint8))
    return int(c), perm


def solve(p, ub0: int = INF, pool: int = 1024, node_budget: int = 0, schedule=None,
          trace_cap: int = 0, ub0_perm=None, init_nodes=None, max_iterations: int = 0,
          export_stack: bool = False, bound: int = 0):
    """Serial pool-synchronous depth-first B&B (Sec. II-A operators, Sec. III pool).

    Returns a dict with status, cmax, perm (None if no schedule beat ub0 and no
    ub0_perm was given), the counters of STATS and, if trace_cap > 0, the
    per-iteration trace rows (parents, children, survivors, UB after).
    init_nodes (uint8 [count, stride] records) replaces the root as the starting
    stack; export_stack returns the stack left at the end under "stack".
    """
    p, n, m = _inst(p)
    perm = np.zeros(n, np.uint8)
    stats = np.zeros(len(STATS), np.int64)
    cmax = ctypes.c_int32(0)
    sched = None if schedule is None else np.ascontiguousarray(schedule, dtype=np.int64)
    trace = np.zeros((max(trace_cap, 1), 4), np.int64)
    stride = (n + 1 + 15) // 16 * 16
    init = None
    if init_nodes is not None:
        init = np.ascontiguousarray(init_nodes, dtype=np.uint8)
        stride = init.shape[1]
    out_count = ctypes.c_int64(0)
    args = [n, m, _p(p, ctypes.c_int32), int(ub0), int(pool), int(node_budget),
            None if sched is None else _p(sched, ctypes.c_int64), 0 if sched is None else len(sched),
            None if init is None else _p(init, ctypes.c_uint8), 0 if init is None else len(init),
            stride, int(max_iterations), ctypes.byref(cmax), _p(perm, ctypes.c_uint8),
            _p(stats, ctypes.c_int64), _p(trace, ctypes.c_int64) if trace_cap > 0 else None,
            int(trace_cap), None, 0, ctypes.byref(out_count), int(bound)]
    rc = _load().orc_solve(*args)
    if rc == ERR_ARG:
        raise ValueError("orc_solve: invalid arguments or init node")
    if rc < 0:
        raise RuntimeError(f"orc_solve failed ({rc})")
    stack = None
    if export_stack:  # second run with a buffer of the right size (the search is deterministic)
        stack = np.zeros((int(out_count.value), stride), np.uint8)
        stats2 = np.zeros(len(STATS), np.int64)
        args[13] = _p(np.zeros(n, np.uint8), ctypes.c_uint8)
        args[14] = _p(stats2, ctypes.c_int64)
        args[15], args[16] = None, 0
        args[17], args[18] = _p(stack, ctypes.c_uint8), len(stack)
        _load().orc_solve(*args)
    res = {k: int(v) for k, v in zip(STATS, stats)}
    res["status"] = int(rc)
    res["cmax"] = int(cmax.value)
    if res["incumbent_updates"] > 0:
        res["perm"] = perm
    else:
        res["perm"] = None if ub0_perm is None else np.asarray(ub0_perm, np.uint8)
    if trace_cap > 0:
        res["trace"] = trace[: min(res["iterations"], trace_cap)].copy()
    res["stack_left"] = int(out_count.value)
    if export_stack:
        res["stack"] = stack
    return res


# --------------------------------------------------------------------------
# Bidirectional branching (fsp_oracle.c, orc_*2 / orc_solve_bidir): a node is
# a prefix perm[:d1], a suffix perm[n-d2:] and the remaining set between them.
# --------------------------------------------------------------------------
def stride2(n: int) -> int:
    """Bytes of a bidirectional record: perm, d1, d2, padded to 16."""
    return (n + 2 + 15) // 16 * 16


def bound_pool2(p, nodes) -> np.ndarray:
    """The bidirectional bound of every record (uint8 [count, stride]: perm[n],
    d1 at byte n, d2 at byte n+1)."""
    p, n, m = _inst(p)
    nodes = np.ascontiguousarray(nodes, dtype=np.uint8)
    count, stride = nodes.shape
    out = np.zeros(count, np.int32)
    rc = _load().orc_bound_pool2(n, m, _p(p, ctypes.c_int32), _p(nodes, ctypes.c_uint8), count, stride,
                                 _p(out, ctypes.c_int32))
    if rc != OK:
        raise ValueError(f"orc_bound_pool2 failed ({rc})")
    return out


def lb2_parts(p, perm, d1: int, d2: int):
    """(LB, LB1, [LB_kl per pair], [D_k per machine]) of one bidirectional node."""
    p, n, m = _inst(p)
    perm = np.ascontiguousarray(perm, dtype=np.uint8)
    lb, lb1 = ctypes.c_int32(0), ctypes.c_int32(0)
    pv = np.zeros(max(num_pairs(m), 1), np.int32)
    D = np.zeros(m, np.int32)
    rc = _load().orc_lb2_parts(n, m, _p(p, ctypes.c_int32), _p(perm, ctypes.c_uint8), int(d1), int(d2),
                               ctypes.byref(lb), ctypes.byref(lb1), _p(pv, ctypes.c_int32), _p(D, ctypes.c_int32))
    if rc != OK:
        raise ValueError("invalid node")
    return int(lb.value), int(lb1.value), pv[: num_pairs(m)], D


def solve_bidir(p, ub0: int = INF, pool: int = 1024, node_budget: int = 0, max_iterations: int = 0,
                trace_cap: int = 0):
    """Pool-synchronous depth-first B&B with bidirectional branching (the
    ends alternate: forward when d1 <= d2).  Same result dict as solve()."""
    p, n, m = _inst(p)
    perm = np.zeros(n, np.uint8)
    stats = np.zeros(len(STATS), np.int64)
    cmax = ctypes.c_int32(0)
    trace = np.zeros((max(trace_cap, 1), 4), np.int64)
    rc = _load().orc_solve_bidir(n, m, _p(p, ctypes.c_int32), int(ub0), int(pool), int(node_budget),
                                 int(max_iterations), ctypes.byref(cmax), _p(perm, ctypes.c_uint8),
                                 _p(stats, ctypes.c_int64), _p(trace, ctypes.c_int64) if trace_cap > 0 else None,
                                 int(trace_cap))
    if rc < 0:
        raise RuntimeError(f"orc_solve_bidir failed ({rc})")
    res = {k: int(v) for k, v in zip(STATS, stats)}
    res["status"] = int(rc)
    res["cmax"] = int(cmax.value)
    res["perm"] = perm.copy() if res["incumbent_updates"] > 0 else None
    if trace_cap > 0:
        res["trace"] = trace[: min(res["iterations"], trace_cap)].copy()
    return res
