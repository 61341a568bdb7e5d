"""Thin Python binding of the C ABI declared in ``include/fsp.h``.

Argument marshalling only: every step of the bounding and the search runs in
the CUDA kernels of ``_build/libfsp.so``.  PyTorch supplies device memory
(tensors' ``data_ptr()``) and streams (``torch.cuda.current_stream()``).  The
library must have been built (``paper_1206_4973_gb300.build.build()``); there
is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, INCOMPLETE = 0, 1
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_CAPACITY, ERR_TIMEOUT = -1, -2, -3, -4, -5
UB_INF = 2**31 - 1
LB_INVALID = -1
_NAMES = {ERR_ARG: "FSP_ERR_ARG", ERR_CUDA: "FSP_ERR_CUDA", ERR_OOM: "FSP_ERR_OOM",
          ERR_CAPACITY: "FSP_ERR_CAPACITY", ERR_TIMEOUT: "FSP_ERR_TIMEOUT"}

# Every symbol include/fsp.h declares.
EXPORTS = ("fsp_default_options", "fsp_node_stride", "fsp_node_stride_bidir", "fsp_bound_pool_bidir",
           "fsp_create_instance", "fsp_destroy_instance",
           "fsp_instance_tables", "fsp_bound_pool", "fsp_check_status", "fsp_solve_workspace_bytes",
           "fsp_solve", "fsp_solve_noalloc", "fsp_neh", "fsp_tune_simulate", "fsp_block_tune_simulate",
           "fsp_node_features",
           "fsp_mlp_create", "fsp_mlp_destroy", "fsp_mlp_num_params", "fsp_mlp_get_params",
           "fsp_mlp_set_params", "fsp_mlp_forward", "fsp_mlp_loss_grad", "fsp_mlp_train_step",
           "fsp_pair_order", "fsp_batch_create", "fsp_batch_destroy", "fsp_batch_run", "fsp_batch_results",
           "fsp_batch_tune_pools", "fsp_batch_set_split", "fsp_batch_set_bidir", "fsp_batch_set_warps",
           "fsp_batch_set_test_hold", "fsp_batch_tune_warps", "fsp_batch_class_stats", "fsp_set_bound", "fsp_instance_host_objects",
           "fsp_last_error")
BOUND_BASE, BOUND_HEADS = 0, 1
SCORE_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int64, ctypes.c_void_p)
NOALLOC_SCRATCH_BYTES = 16 << 20


class FspError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class fsp_stats(ctypes.Structure):
    _fields_ = [("nodes_bounded", ctypes.c_int64), ("nodes_branched", ctypes.c_int64),
                ("nodes_pruned", ctypes.c_int64), ("leaves", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("incumbent_updates", ctypes.c_int64),
                ("time_ms", ctypes.c_double), ("select_ms", ctypes.c_double),
                ("bound_ms", ctypes.c_double), ("compact_ms", ctypes.c_double),
                ("tuned_pool", ctypes.c_int64), ("early_pruned", ctypes.c_int64), ("infer_ms", ctypes.c_double),
                ("tuned_warps", ctypes.c_int64), ("families_closed_lb1", ctypes.c_int64),
                ("families_closed_predicted", ctypes.c_int64), ("exact_pair_evals", ctypes.c_int64)]


class fsp_options(ctypes.Structure):
    _fields_ = [("pool_size", ctypes.c_int64), ("node_budget", ctypes.c_int64),
                ("stack_capacity", ctypes.c_int64), ("ub0_perm", ctypes.POINTER(ctypes.c_int32)),
                ("trace", ctypes.POINTER(ctypes.c_int64)), ("trace_cap", ctypes.c_int64),
                ("schedule", ctypes.POINTER(ctypes.c_int64)), ("schedule_len", ctypes.c_int64),
                ("workspace", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("init_nodes", ctypes.c_void_p), ("init_count", ctypes.c_int64),
                ("max_iterations", ctypes.c_int64), ("out_nodes", ctypes.c_void_p),
                ("out_cap", ctypes.c_int64), ("out_count", ctypes.POINTER(ctypes.c_int64)),
                ("profile", ctypes.c_int), ("tune_window", ctypes.c_int64),
                ("schedule_out", ctypes.POINTER(ctypes.c_int64)), ("schedule_out_cap", ctypes.c_int64),
                ("order", ctypes.c_int), ("topk", ctypes.c_int), ("model", ctypes.c_void_p),
                ("log_nodes", ctypes.c_void_p), ("log_cap", ctypes.c_int64),
                ("log_count", ctypes.POINTER(ctypes.c_int64)), ("log_lbs", ctypes.c_void_p),
                ("branching", ctypes.c_int), ("warps", ctypes.c_int)]
ORDER_PLAIN, ORDER_LEARNED = 0, 1
BRANCH_FORWARD, BRANCH_BIDIR = 0, 1


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfsp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "paper_1206_4973_gb300.build.build() (no fallback exists)")
    L = ctypes.CDLL(path)
    vp, i32p, u8p, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint8), ctypes.c_int64
    sig = {
        "fsp_default_options": (ctypes.c_int, [ctypes.POINTER(fsp_options)]),
        "fsp_node_stride": (ctypes.c_int, [ctypes.c_int]),
        "fsp_node_stride_bidir": (ctypes.c_int, [ctypes.c_int]),
        "fsp_bound_pool_bidir": (ctypes.c_int, [vp, vp, i64, vp, vp]),
        "fsp_create_instance": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, i32p, ctypes.POINTER(vp)]),
        "fsp_destroy_instance": (None, [vp]),
        "fsp_instance_tables": (ctypes.c_int, [vp, i32p, i32p, u8p]),
        "fsp_bound_pool": (ctypes.c_int, [vp, vp, i64, ctypes.c_int32, vp, vp]),
        "fsp_check_status": (ctypes.c_int, [vp, vp]),
        "fsp_solve_workspace_bytes": (i64, [vp, ctypes.POINTER(fsp_options)]),
        "fsp_solve": (ctypes.c_int, [vp, ctypes.c_int32, i32p, vp, ctypes.POINTER(fsp_stats),
                                     ctypes.POINTER(fsp_options)]),
        "fsp_solve_noalloc": (ctypes.c_int, [vp, ctypes.c_int32, i32p, vp, ctypes.POINTER(fsp_stats),
                                             ctypes.POINTER(fsp_options)]),
        "fsp_neh": (ctypes.c_int, [vp, i32p, i32p]),
        "fsp_tune_simulate": (i64, [i64, ctypes.c_int, i64, SCORE_FN, vp, ctypes.POINTER(ctypes.c_int64), i64,
                                    ctypes.POINTER(ctypes.c_int64)]),
        "fsp_block_tune_simulate": (i64, [ctypes.c_int, i64, SCORE_FN, vp, ctypes.POINTER(ctypes.c_int64), i64,
                                          ctypes.POINTER(ctypes.c_int64)]),
        "fsp_node_features": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
        "fsp_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.POINTER(vp)]),
        "fsp_mlp_destroy": (None, [vp]),
        "fsp_mlp_num_params": (i64, [vp]),
        "fsp_mlp_get_params": (ctypes.c_int, [vp, vp]),
        "fsp_mlp_set_params": (ctypes.c_int, [vp, vp]),
        "fsp_mlp_forward": (ctypes.c_int, [vp, vp, i64, vp, vp]),
        "fsp_mlp_loss_grad": (ctypes.c_int, [vp, vp, vp, i64, ctypes.POINTER(ctypes.c_float), vp, vp]),
        "fsp_mlp_train_step": (ctypes.c_int, [vp, vp, vp, i64, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                              vp]),
        "fsp_pair_order": (ctypes.c_int, [vp, vp, vp, i64, ctypes.c_int, vp, vp]),
        "fsp_batch_create": (ctypes.c_int, [ctypes.c_int, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "fsp_batch_destroy": (None, [vp]),
        "fsp_batch_run": (ctypes.c_int, [vp, vp]),
        "fsp_batch_results": (ctypes.c_int, [vp, vp, vp, vp]),
        "fsp_batch_tune_pools": (ctypes.c_int, [ctypes.c_int, vp, vp, i64, vp]),
        "fsp_batch_set_split": (ctypes.c_int, [vp, ctypes.c_int]),
        "fsp_batch_set_bidir": (ctypes.c_int, [vp, ctypes.c_int]),
        "fsp_batch_set_test_hold": (ctypes.c_int, [vp, ctypes.c_int]),
        "fsp_batch_set_warps": (ctypes.c_int, [vp, vp]),
        "fsp_batch_tune_warps": (ctypes.c_int, [ctypes.c_int, vp, vp, vp, i64, vp]),
        "fsp_batch_class_stats": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "fsp_set_bound": (ctypes.c_int, [vp, ctypes.c_int]),
        "fsp_instance_host_objects": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64),
                                                     ctypes.POINTER(ctypes.c_int64)]),
        "fsp_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int) -> int:
    if rc < 0:
        raise FspError(rc, load().fsp_last_error().decode())
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Instance:
    """Handle of a device-resident instance (processing times + tables)."""

    def __init__(self, handle, n: int, m: int):
        self.handle, self.n, self.m = handle, n, m
        self.stride = fsp_node_stride(n)

    def set_bound(self, variant: int) -> None:
        """BOUND_BASE or BOUND_HEADS (release times raised by the smallest heads)."""
        _check(load().fsp_set_bound(self.handle, int(variant)))
        self.bound = int(variant)

    def close(self):
        if self.handle:
            fsp_destroy_instance(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fsp_node_stride(n: int) -> int:
    return int(load().fsp_node_stride(int(n)))


def fsp_create_instance(p) -> Instance:
    """p: n x m int32 processing times (job-major), host array-like."""
    p = np.ascontiguousarray(np.asarray(p), dtype=np.int32)
    if p.ndim != 2:
        raise ValueError("p must be n x m")
    n, m = p.shape
    h = ctypes.c_void_p()
    _check(load().fsp_create_instance(n, m, p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      ctypes.byref(h)))
    return Instance(h, n, m)


def fsp_destroy_instance(inst: Instance) -> None:
    if inst.handle:
        load().fsp_destroy_instance(inst.handle)
        inst.handle = None


def fsp_instance_tables(inst: Instance):
    P = inst.m * (inst.m - 1) // 2
    q = np.zeros((inst.n, inst.m), np.int32)
    lag = np.zeros((P, inst.n), np.int32)
    order = np.zeros((P, inst.n), np.uint8)
    _check(load().fsp_instance_tables(inst.handle, q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      lag.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      order.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return q, lag, order


def fsp_bound_pool(inst: Instance, nodes, ub: int = UB_INF, lb_out=None, stream=None, count=None):
    """Bound node records (CUDA uint8 tensor [count, stride]) into lb_out
    (CUDA int32 tensor [count]; allocated when None).  Asynchronous."""
    import torch
    if count is None:
        count = nodes.shape[0]
    if lb_out is None:
        lb_out = torch.empty(count, dtype=torch.int32, device=nodes.device)
    if nodes.dtype != torch.uint8 or not nodes.is_cuda or not lb_out.is_cuda or lb_out.dtype != torch.int32:
        raise ValueError("nodes must be a CUDA uint8 tensor and lb_out a CUDA int32 tensor")
    if not nodes.is_contiguous() or not lb_out.is_contiguous():
        raise ValueError("nodes and lb_out must be contiguous")
    if count and (nodes.numel() < count * inst.stride or lb_out.numel() < count):
        raise ValueError("buffers smaller than count records")
    _check(load().fsp_bound_pool(inst.handle, nodes.data_ptr(), int(count), int(ub), lb_out.data_ptr(),
                                 _stream(stream)))
    return lb_out


def fsp_node_stride_bidir(n: int) -> int:
    return int(load().fsp_node_stride_bidir(int(n)))


def fsp_bound_pool_bidir(inst: Instance, nodes, lb_out=None, stream=None, count=None):
    """Bound bidirectional records (CUDA uint8 tensor [count, fsp_node_stride_bidir(n)]:
    perm, d1 at byte n, d2 at byte n+1) into lb_out (CUDA int32 [count]).  Asynchronous."""
    import torch
    if count is None:
        count = nodes.shape[0]
    if lb_out is None:
        lb_out = torch.empty(count, dtype=torch.int32, device=nodes.device)
    if nodes.dtype != torch.uint8 or not nodes.is_cuda or not lb_out.is_cuda or lb_out.dtype != torch.int32:
        raise ValueError("nodes must be a CUDA uint8 tensor and lb_out a CUDA int32 tensor")
    if not nodes.is_contiguous() or not lb_out.is_contiguous():
        raise ValueError("nodes and lb_out must be contiguous")
    if count and (nodes.numel() < count * fsp_node_stride_bidir(inst.n) or lb_out.numel() < count):
        raise ValueError("buffers smaller than count records")
    _check(load().fsp_bound_pool_bidir(inst.handle, nodes.data_ptr(), int(count), lb_out.data_ptr(),
                                       _stream(stream)))
    return lb_out


def fsp_check_status(inst: Instance, stream=None) -> None:
    _check(load().fsp_check_status(inst.handle, _stream(stream)))


def _ptr(buf):
    """Address of a torch tensor (device or host) or a numpy array."""
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr()
    return np.asarray(buf).ctypes.data


def fsp_instance_host_objects(inst: Instance):
    """(pinned read-back blocks, CUDA events) the instance has created so far."""
    pb, ev = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().fsp_instance_host_objects(inst.handle, ctypes.byref(pb), ctypes.byref(ev)))
    return int(pb.value), int(ev.value)


def fsp_neh(inst: Instance):
    """NEH on the device: (makespan, permutation as int32 array)."""
    perm = np.zeros(inst.n, np.int32)
    c = ctypes.c_int32(0)
    _check(load().fsp_neh(inst.handle, ctypes.byref(c), perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return int(c.value), perm


def fsp_tune_simulate(nodes_per_cta: int, sms: int, max_pool: int, score):
    """Run the pool tuner against score(pool) -> float; returns (pools tried, best)."""
    cb = SCORE_FN(lambda pool, _u: float(score(int(pool))))
    out = np.zeros(64, np.int64)
    best = ctypes.c_int64(0)
    k = _check(int(load().fsp_tune_simulate(int(nodes_per_cta), int(sms), int(max_pool), cb, None,
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 64,
                                            ctypes.byref(best))))
    return out[:k].tolist(), int(best.value)


def fsp_block_tune_simulate(ncand: int, window: int, score):
    """Run the block-shape tuner against score(cand) -> nodes per iteration;
    returns (candidate of every iteration, kept candidate)."""
    cb = SCORE_FN(lambda cand, _u: float(score(int(cand))))
    out = np.zeros(4096, np.int64)
    best = ctypes.c_int64(0)
    k = _check(int(load().fsp_block_tune_simulate(int(ncand), int(window), cb, None,
                                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 4096,
                                                  ctypes.byref(best))))
    return out[:k].tolist(), int(best.value)


_default_options = None  # fsp_default_options' struct, as bytes


def _options(pool_size=1024, node_budget=0, stack_capacity=0, ub0_perm=None, trace_cap=0,
             schedule=None, stream=None, init_nodes=None, init_count=None, max_iterations=0,
             out_nodes=None, profile=False, tune_window=0, schedule_out=None, model=None, topk=0,
             log_nodes=None, log_lbs=None, branching=0, warps=0):
    global _default_options
    if _default_options is None:
        d = fsp_options()
        load().fsp_default_options(ctypes.byref(d))
        _default_options = bytes(d)
    o = fsp_options.from_buffer_copy(_default_options)
    o.pool_size = int(pool_size)
    o.tune_window = int(tune_window)
    o.branching = int(branching)
    o.warps = int(warps)
    if model is not None:
        o.order = ORDER_LEARNED
        o.model = model.handle
        o.topk = int(topk)
    o.node_budget = int(node_budget)
    o.stack_capacity = int(stack_capacity)
    o.max_iterations = int(max_iterations)
    o.profile = 1 if profile else 0
    keep = []
    if init_nodes is not None:
        if not hasattr(init_nodes, "data_ptr"):
            init_nodes = np.ascontiguousarray(init_nodes, dtype=np.uint8)
        keep.append(init_nodes)
        o.init_nodes = _ptr(init_nodes)
        o.init_count = int(init_nodes.shape[0] if init_count is None else init_count)
    if schedule_out is not None:
        keep.append(schedule_out)
        o.schedule_out = schedule_out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        o.schedule_out_cap = len(schedule_out)
    out_count = ctypes.c_int64(0)
    keep.append(out_count)
    log_count = ctypes.c_int64(0)
    keep.append(log_count)
    o.log_count = ctypes.pointer(log_count)
    if log_nodes is not None:
        keep.append(log_nodes)
        o.log_nodes = log_nodes.data_ptr()
        o.log_cap = int(log_nodes.shape[0])
        if log_lbs is not None:
            if log_lbs.numel() < o.log_cap:
                raise ValueError("log_lbs needs an entry per log_nodes record")
            keep.append(log_lbs)
            o.log_lbs = log_lbs.data_ptr()
    o.out_count = ctypes.pointer(out_count)
    if out_nodes is not None:
        keep.append(out_nodes)
        o.out_nodes = _ptr(out_nodes)
        o.out_cap = int(out_nodes.shape[0])
    if ub0_perm is not None:
        a = np.ascontiguousarray(ub0_perm, dtype=np.int32)
        keep.append(a)
        o.ub0_perm = a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    trace = None
    if trace_cap > 0:
        trace = np.zeros((trace_cap, 4), np.int64)
        keep.append(trace)
        o.trace = trace.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        o.trace_cap = trace_cap
    if schedule is not None:
        s = np.ascontiguousarray(schedule, dtype=np.int64)
        keep.append(s)
        o.schedule = s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        o.schedule_len = len(s)
    o.stream = _stream(stream)
    o._log_count = log_count
    return o, keep, trace, out_count


def fsp_solve_workspace_bytes(inst: Instance, **kw) -> int:
    o, _keep, _, _ = _options(**kw)
    return _check(int(load().fsp_solve_workspace_bytes(inst.handle, ctypes.byref(o))))


STATS = ("nodes_bounded", "nodes_branched", "nodes_pruned", "leaves", "iterations", "incumbent_updates")
_RESULT_FIELDS = STATS + ("time_ms", "select_ms", "bound_ms", "compact_ms", "infer_ms", "tuned_pool", "tuned_warps",
                          "early_pruned", "families_closed_lb1", "families_closed_predicted", "exact_pair_evals")


def fsp_solve(inst: Instance, ub0: int = UB_INF, pool_size: int = 1024, node_budget: int = 0,
              stack_capacity: int = 0, ub0_perm=None, trace_cap: int = 0, schedule=None, stream=None,
              workspace=None, init_nodes=None, init_count=None, max_iterations: int = 0,
              out_nodes=None, profile: bool = False, tune_window: int = 0, schedule_cap: int = 0,
              model=None, topk: int = 0, log_nodes=None, log_lbs=None, branching: int = BRANCH_FORWARD,
              warps: int = 0):
    """Exact B&B on the device.  The scratch is a torch uint8 tensor (allocated
    here when `workspace` is None).  init_nodes (host array or device tensor of
    records) starts the search from that stack; out_nodes (host array or
    device tensor [cap, stride]) receives the stack left at the end.  Returns a
    dict: status, cmax, perm (None if the search found nothing better than ub0
    and no ub0_perm was given), the counters of STATS, time_ms, the phase
    times when profile is set, stack_left and, if trace_cap > 0, the trace."""
    import torch
    sched_out = np.zeros(schedule_cap, np.int64) if schedule_cap > 0 else None
    o, keep, trace, out_count = _options(pool_size, node_budget, stack_capacity, ub0_perm, trace_cap,
                                         schedule, stream, init_nodes, init_count, max_iterations,
                                         out_nodes, profile, tune_window, sched_out, model, topk, log_nodes,
                                         log_lbs, branching, warps)
    nbytes = _check(int(load().fsp_solve_workspace_bytes(inst.handle, ctypes.byref(o))))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    elif workspace.numel() < nbytes:
        raise ValueError(f"workspace needs {nbytes} bytes")
    o.workspace = workspace.data_ptr()
    perm = np.empty(inst.n, np.int32)
    perm.fill(-1)
    cmax = ctypes.c_int32(0)
    st = fsp_stats()
    rc = _check(load().fsp_solve(inst.handle, int(ub0), ctypes.byref(cmax), perm.ctypes.data, ctypes.byref(st),
                                 ctypes.byref(o)))
    # ctypes returns the struct's integer and floating fields as Python ints and floats
    res = {k: getattr(st, k) for k in _RESULT_FIELDS}
    res["stack_left"] = out_count.value
    res["status"] = rc
    res["cmax"] = cmax.value
    res["perm"] = perm if perm[0] >= 0 else None
    res["logged"] = o._log_count.value
    if trace is not None:
        res["trace"] = trace[: min(res["iterations"], trace_cap)].copy()
    if sched_out is not None:
        res["schedule"] = sched_out[: min(res["iterations"], schedule_cap)].copy()
    del keep
    return res


class SolveCall:
    """A prepared fsp_solve: the options struct, the workspace (allocated here
    when None) and the result buffers are built once, so a repeated call with
    the same arguments costs only the call into the library.  run() returns
    the dict fsp_solve returns (without trace and schedule)."""

    def __init__(self, inst: Instance, ub0: int = UB_INF, workspace=None, **kw):
        import torch
        self.inst, self.ub0 = inst, int(ub0)
        self.o, self._keep, _trace, self._out_count = _options(**kw)
        nbytes = _check(int(load().fsp_solve_workspace_bytes(inst.handle, ctypes.byref(self.o))))
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        elif workspace.numel() < nbytes:
            raise ValueError(f"workspace needs {nbytes} bytes")
        self.workspace = workspace
        self.o.workspace = workspace.data_ptr()
        self.perm = np.empty(inst.n, np.int32)
        self._cmax = ctypes.c_int32(0)
        self._st = fsp_stats()
        self._args = (inst.handle, self.ub0, ctypes.byref(self._cmax), self.perm.ctypes.data,
                      ctypes.byref(self._st), ctypes.byref(self.o))
        self._fn = load().fsp_solve

    def run(self) -> dict:
        self.perm.fill(-1)
        rc = _check(self._fn(*self._args))
        st = self._st
        res = {k: getattr(st, k) for k in _RESULT_FIELDS}
        res["stack_left"] = self._out_count.value
        res["status"] = rc
        res["cmax"] = self._cmax.value
        res["perm"] = self.perm if self.perm[0] >= 0 else None
        return res


def fsp_solve_noalloc(inst: Instance, ub0: int = UB_INF, pool_size: int = 1024, node_budget: int = 0,
                      stack_capacity: int = 0, ub0_perm=None, trace_cap: int = 0, schedule=None, stream=None,
                      init_nodes=None, init_count=None, max_iterations: int = 0, out_nodes=None):
    """fsp_solve through the entry point that allocates no device memory (its
    scratch is the library's fixed array of NOALLOC_SCRATCH_BYTES).  For
    callers that cannot allocate during a call; overlapping calls race on the
    shared array, so serialise them.  Same results as fsp_solve, times 0."""
    o, keep, trace, out_count = _options(pool_size, node_budget, stack_capacity, ub0_perm, trace_cap,
                                         schedule, stream, init_nodes, init_count, max_iterations,
                                         out_nodes, False)
    perm = np.full(inst.n, -1, np.int32)
    cmax = ctypes.c_int32(0)
    st = fsp_stats()
    rc = _check(load().fsp_solve_noalloc(inst.handle, int(ub0), ctypes.byref(cmax), perm.ctypes.data,
                                         ctypes.byref(st), ctypes.byref(o)))
    res = {k: int(getattr(st, k)) for k in STATS}
    res["status"] = rc
    res["cmax"] = int(cmax.value)
    res["perm"] = perm if perm[0] >= 0 else None
    res["stack_left"] = int(out_count.value)
    if trace is not None:
        res["trace"] = trace[: min(res["iterations"], trace_cap)].copy()
    del keep
    return res


# ------------------------------------------------------------ learned order --

def fsp_node_features(inst: Instance, nodes, x=None, label=None, stream=None):
    """Features (CUDA float32 [count, 2m+1]) and labels (CUDA int32 [count]) of
    node records (CUDA uint8 [count, stride])."""
    import torch
    count = nodes.shape[0]
    F = 2 * inst.m + 1
    if x is None:
        x = torch.empty((count, F), dtype=torch.float32, device=nodes.device)
    if label is None:
        label = torch.empty(count, dtype=torch.int32, device=nodes.device)
    _check(load().fsp_node_features(inst.handle, nodes.data_ptr(), count, x.data_ptr(), label.data_ptr(),
                                    _stream(stream)))
    return x, label


class Mlp:
    """Handle of a device-resident pair-scoring network."""

    def __init__(self, in_dim: int, hidden: int, out_dim: int, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().fsp_mlp_create(int(in_dim), int(hidden), int(out_dim), int(seed), ctypes.byref(h)))
        self.handle, self.F, self.H, self.P = h, in_dim, hidden, out_dim

    def close(self):
        if self.handle:
            load().fsp_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self) -> int:
        return int(load().fsp_mlp_num_params(self.handle))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params(), np.float32)
        _check(load().fsp_mlp_get_params(self.handle, out.ctypes.data))
        return out

    def set_params(self, w) -> None:
        w = np.ascontiguousarray(w, dtype=np.float32)
        if w.size != self.num_params():
            raise ValueError("wrong number of parameters")
        _check(load().fsp_mlp_set_params(self.handle, w.ctypes.data))

    def split(self, flat):
        """Flat parameters -> dict W1, b1, W2, b2, W3, b3 (numpy views)."""
        F, H, P = self.F, self.H, self.P
        o, out = 0, {}
        for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, P)),
                            ("b3", (P,))):
            size = int(np.prod(shape))
            out[name] = flat[o:o + size].reshape(shape)
            o += size
        return out

    def forward(self, X, scores=None, stream=None):
        import torch
        if scores is None:
            scores = torch.empty((X.shape[0], self.P), dtype=torch.float32, device=X.device)
        _check(load().fsp_mlp_forward(self.handle, X.data_ptr(), X.shape[0], scores.data_ptr(), _stream(stream)))
        return scores

    def loss_grad(self, X, y, stream=None):
        import torch
        g = torch.empty(self.num_params(), dtype=torch.float32, device=X.device)
        loss = ctypes.c_float(0)
        _check(load().fsp_mlp_loss_grad(self.handle, X.data_ptr(), y.data_ptr(), X.shape[0], ctypes.byref(loss),
                                        g.data_ptr(), _stream(stream)))
        return float(loss.value), g

    def train_step(self, X, y, lr: float, stream=None) -> float:
        loss = ctypes.c_float(0)
        _check(load().fsp_mlp_train_step(self.handle, X.data_ptr(), y.data_ptr(), X.shape[0], float(lr),
                                         ctypes.byref(loss), _stream(stream)))
        return float(loss.value)


def fsp_pair_order(inst: Instance, mlp: Mlp, nodes, k: int = 4, stream=None):
    """The k best-scored pairs of each node record (CUDA uint8 [count, stride]):
    CUDA int16 [count, k], best first."""
    import torch
    out = torch.empty((nodes.shape[0], k), dtype=torch.int16, device=nodes.device)
    _check(load().fsp_pair_order(inst.handle, mlp.handle, nodes.data_ptr(), nodes.shape[0], int(k), out.data_ptr(),
                                 _stream(stream)))
    return out


# ------------------------------------------------------------------ batches --

class fsp_batch_result(ctypes.Structure):
    _fields_ = [("cmax", ctypes.c_int32), ("status", ctypes.c_int32), ("nodes_bounded", ctypes.c_int64),
                ("nodes_branched", ctypes.c_int64), ("nodes_pruned", ctypes.c_int64), ("leaves", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("incumbent_updates", ctypes.c_int64), ("pool", ctypes.c_int64)]


class fsp_batch_class_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("warps", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("instances", ctypes.c_int32), ("items", ctypes.c_int32), ("donated", ctypes.c_int32),
                ("busy_mean_ms", ctypes.c_double),
                ("busy_min_ms", ctypes.c_double), ("busy_max_ms", ctypes.c_double),
                ("first_start_ms", ctypes.c_double), ("last_end_ms", ctypes.c_double),
                ("launch_span_ms", ctypes.c_double)]


def _flatten(instances):
    shapes = np.array([[p.shape[0], p.shape[1]] for p in instances], dtype=np.int32)
    flat = np.concatenate([np.ascontiguousarray(p, dtype=np.int32).ravel() for p in instances]).astype(np.int32)
    return shapes, flat


def fsp_batch_tune_pools(instances, probe_budget: int = 200000):
    """Pool size per shape on measured throughput; returns one pool per instance."""
    shapes, flat = _flatten(instances)
    out = np.zeros(len(instances), np.int64)
    _check(load().fsp_batch_tune_pools(len(instances), shapes.ctypes.data, flat.ctypes.data, int(probe_budget),
                                       out.ctypes.data))
    return out


def fsp_batch_tune_warps(instances, pools, probe_budget: int = 200000):
    """Block shape (warps per CTA) per shape on measured throughput; returns one per instance."""
    shapes, flat = _flatten(instances)
    pools = np.ascontiguousarray(pools, dtype=np.int64)
    out = np.zeros(len(instances), np.int32)
    _check(load().fsp_batch_tune_warps(len(instances), shapes.ctypes.data, flat.ctypes.data, pools.ctypes.data,
                                       int(probe_budget), out.ctypes.data))
    return out


class Batch:
    """Instances of mixed shape solved in one persistent launch (a CUDA graph)."""

    def __init__(self, instances, pools, budgets=None, ub0=None, split=False, warps=None):
        shapes, flat = _flatten(instances)
        self.count = len(instances)
        self.n = shapes[:, 0].copy()
        pools = np.ascontiguousarray(pools, dtype=np.int64)
        bud = None if budgets is None else np.ascontiguousarray(budgets, dtype=np.int64)
        ub = None if ub0 is None else np.ascontiguousarray(ub0, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(load().fsp_batch_create(self.count, shapes.ctypes.data, flat.ctypes.data, pools.ctypes.data,
                                       None if bud is None else bud.ctypes.data,
                                       None if ub is None else ub.ctypes.data, ctypes.byref(h)))
        self.handle = h
        if warps is not None:
            self.set_warps(warps)
        if split:
            self.set_split(True)

    def set_warps(self, warps):
        """Warps per CTA for each instance (fsp_batch_set_warps; None = 8 for all)."""
        if warps is None:
            _check(load().fsp_batch_set_warps(self.handle, None))
            return
        w = np.ascontiguousarray(warps, dtype=np.int32)
        if w.shape != (self.count,):
            raise ValueError("one block shape per instance")
        _check(load().fsp_batch_set_warps(self.handle, w.ctypes.data))

    def set_split(self, on: bool):
        """Work items = the subtrees of the roots (fsp_batch_set_split)."""
        _check(load().fsp_batch_set_split(self.handle, 1 if on else 0))

    def set_bidir(self, on: bool):
        """Bidirectional branching for every instance (fsp_batch_set_bidir)."""
        _check(load().fsp_batch_set_bidir(self.handle, 1 if on else 0))

    def set_test_hold(self, on: bool):
        """Test hook: every wait on the split mode's donations runs out
        (fsp_batch_set_test_hold)."""
        _check(load().fsp_batch_set_test_hold(self.handle, 1 if on else 0))

    def close(self):
        if self.handle:
            load().fsp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, stream=None):
        _check(load().fsp_batch_run(self.handle, _stream(stream)))

    def class_stats(self):
        """Per class (shape, warps) of the last run: CTAs, items and CTA lifetimes (fsp_batch_class_stats)."""
        count = ctypes.c_int(0)
        _check(load().fsp_batch_class_stats(self.handle, None, 0, ctypes.byref(count)))
        arr = (fsp_batch_class_info * max(1, count.value))()
        _check(load().fsp_batch_class_stats(self.handle, ctypes.addressof(arr), count.value, ctypes.byref(count)))
        return [{k: getattr(arr[i], k) for k, _ in fsp_batch_class_info._fields_} for i in range(count.value)]

    def results(self, stream=None):
        res = (fsp_batch_result * self.count)()
        perms = np.zeros((self.count, 255), np.int32)
        _check(load().fsp_batch_results(self.handle, ctypes.addressof(res), perms.ctypes.data, _stream(stream)))
        out = []
        for i in range(self.count):
            r = {k: int(getattr(res[i], k)) for k, _ in fsp_batch_result._fields_}
            r["perm"] = perms[i, : self.n[i]].copy()
            out.append(r)
        return out
