"""The family kernel (a parent's children bounded together from the parent's
prefix and suffix maxima per machine pair) gives every child the bound the
oracle computes for it, bit for bit, and runs the same search as the
per-child kernel."""
import os

import numpy as np
import pytest

import oracle
from paper_1206_4973_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("status", "cmax", "nodes_bounded", "nodes_branched", "nodes_pruned", "leaves", "iterations",
        "incumbent_updates", "stack_left")


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_1206_4973_gb300 import build, fsp
    build.build()
    fsp.load()
    assert torch.cuda.is_available()
    return fsp


def per_child(F, inst, **kw):
    os.environ["FSP_FAMILY"] = "0"
    try:
        return F.fsp_solve(inst, **kw)
    finally:
        del os.environ["FSP_FAMILY"]


# shapes across the record widths (16, 32, 48, 64 bytes), the 32-job mask
# boundary, every machine template, one-parent pools and a shape whose
# tables do not fit the family kernel (63 x 20: per-child kernel)
CASES = [(12, 5, 0, 1024), (20, 20, 1, 4096), (15, 10, 3, 512), (31, 20, 5, 2048), (32, 20, 9, 1024),
         (33, 10, 21, 2048), (50, 5, 4, 4096), (63, 10, 8, 2048), (9, 20, 88, 64), (20, 5, 2, 1),
         (63, 20, 12, 512)]


@pytest.mark.parametrize("n,m,seed,pool", CASES)
def test_children_bounds_match_oracle(F, n, m, seed, pool):
    import torch
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst)
    cap = 60000
    log = torch.zeros((cap, inst.stride), dtype=torch.uint8, device="cuda")
    lbs = torch.zeros(cap, dtype=torch.int32, device="cuda")
    r = F.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=pool, node_budget=40000, log_nodes=log, log_lbs=lbs)
    k = r["logged"]
    assert k == min(cap, r["nodes_bounded"]) and k > 0
    rec = log[:k].cpu().numpy()
    got = lbs[:k].cpu().numpy()
    idx = np.unique(np.linspace(0, k - 1, min(k, 15000)).astype(np.int64))
    assert np.array_equal(got[idx], oracle.bound_pool(p, rec[idx]))


@pytest.mark.parametrize("n,m,seed,pool,budget", [(12, 5, 0, 1024, 0), (20, 20, 6, 8192, 200000),
                                                  (50, 10, 7, 4096, 100000), (32, 5, 11, 256, 300000)])
def test_family_and_per_child_kernels_search_alike(F, n, m, seed, pool, budget):
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst)
    kw = dict(ub0=ub0, ub0_perm=perm0, pool_size=pool, node_budget=budget, trace_cap=100000)
    a = F.fsp_solve(inst, **kw)
    b = per_child(F, inst, **kw)
    for key in KEYS:
        assert a[key] == b[key], key
    assert np.array_equal(a["trace"], b["trace"])
    assert (a["perm"] is None) == (b["perm"] is None)
    if a["perm"] is not None:
        assert list(a["perm"]) == list(b["perm"])


@pytest.mark.parametrize("n,m,seed,pool,budget,max_it", [(12, 5, 0, 64, 0, 0), (20, 20, 6, 4096, 150000, 0),
                                                         (20, 10, 5, 0, 300000, 0), (15, 5, 3, 128, 0, 37),
                                                         (50, 5, 3, 2048, 80000, 0)])
def test_launching_ahead_gives_the_same_search(F, n, m, seed, pool, budget, max_it):
    """Iterations launched one ahead of their read-back (the default) and one
    at a time (forced by phase timing) stop at the same budget or iteration
    cap with the same state; pool 0 runs the tuner first."""
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst)
    out_a = np.zeros((60000, inst.stride), np.uint8)
    out_b = np.zeros_like(out_a)
    kw = dict(ub0=ub0, ub0_perm=perm0, pool_size=pool, node_budget=budget, max_iterations=max_it,
              trace_cap=100000, schedule_cap=100000)
    a = F.fsp_solve(inst, out_nodes=out_a, **kw)
    if pool == 0:  # the tuner's choices depend on measured times: replay them
        kw = dict(kw, pool_size=1024, schedule=a["schedule"])
    b = F.fsp_solve(inst, out_nodes=out_b, profile=True, **kw)
    for key in KEYS:
        assert a[key] == b[key], key
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["schedule"], b["schedule"])
    k = min(a["stack_left"], len(out_a))
    assert np.array_equal(out_a[:k], out_b[:k])


def test_block_shape_tuning_reports_a_shape_and_keeps_the_search(F):
    """pool_size = 0 tunes the pool, then the family kernel's warps per CTA;
    the search equals a replay of the tuned pools with the default shape."""
    p = inputs.instance(20, 10, 5)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst)
    a = F.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=0, tune_window=4, schedule_cap=100000,
                    trace_cap=100000)
    b = F.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=1024, schedule=a["schedule"], trace_cap=100000)
    for key in KEYS:
        assert a[key] == b[key], key
    assert np.array_equal(a["trace"], b["trace"])
    most = b["tuned_warps"]  # a fixed pool keeps the most warps that fit (up to 20)
    assert 16 <= most <= 20
    assert a["status"] == F.OK and a["tuned_warps"] in (4, 8, 12, most)


@pytest.mark.parametrize("n,m,seed,count", [(20, 20, 1, 4096), (12, 5, 2, 777), (33, 10, 3, 3000), (50, 20, 4, 1500),
                                            (63, 5, 5, 1)])
def test_small_pools_one_warp_per_node(F, n, m, seed, count):
    """fsp_bound_pool on a small pool (one warp per node) gives the oracle's
    bounds and the per-thread kernel's, also for the heads variant, and flags
    malformed records the same way."""
    import torch
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    rec = inputs.random_prefix_pool(n, count, inputs.SplitMix64(seed + 9))
    rec[::5, n] = n
    rec[1::7, n] = n - 1
    dev = torch.from_numpy(rec).cuda()
    for variant in (F.BOUND_BASE, F.BOUND_HEADS):
        inst.set_bound(variant)
        got = F.fsp_bound_pool(inst, dev).cpu().numpy()
        F.fsp_check_status(inst)
        assert np.array_equal(got, oracle.bound_pool(p, rec, bound=variant))
        os.environ["FSP_FAMILY_POOL0"] = "1"
        try:
            per_thread = F.fsp_bound_pool(inst, dev).cpu().numpy()
        finally:
            del os.environ["FSP_FAMILY_POOL0"]
        assert np.array_equal(got, per_thread)
    if count > 3:
        bad = rec.copy()
        bad[2, 0] = bad[2, 1]          # a repeated job
        bad[3, n] = n + 1              # depth > n
        got = F.fsp_bound_pool(inst, torch.from_numpy(bad).cuda()).cpu().numpy()
        assert got[2] == F.LB_INVALID and got[3] == F.LB_INVALID
        with pytest.raises(F.FspError):
            F.fsp_check_status(inst)
        keep = np.ones(count, bool)
        keep[[2, 3]] = False
        assert np.array_equal(got[keep], oracle.bound_pool(p, rec[keep], bound=F.BOUND_HEADS))


def test_fixed_block_shape_gives_the_same_search(F):
    """fsp_options.warps fixes the bounding kernel's block shape (warps per
    CTA): every shape gives the search of the default shape, counter for
    counter, trace and incumbent; a shape outside 1..20 or too large for the
    tables is refused."""
    p = inputs.instance(20, 20, 6)
    inst = F.fsp_create_instance(p)
    u, perm = F.fsp_neh(inst)
    kw = dict(ub0=u, ub0_perm=perm, pool_size=8192, node_budget=1_000_000, trace_cap=4096)
    ref = F.fsp_solve(inst, **kw)
    for w in (1, 2, 5, 8, 16, 20):
        got = F.fsp_solve(inst, warps=w, **kw)
        for k in ("status", "cmax", "nodes_bounded", "nodes_branched", "nodes_pruned", "leaves", "iterations",
                  "incumbent_updates", "stack_left"):
            assert got[k] == ref[k], (w, k)
        assert np.array_equal(got["trace"], ref["trace"]), w
        assert list(got["perm"]) == list(ref["perm"])
    for w in (-1, 21):
        with pytest.raises(F.FspError):
            F.fsp_solve(inst, warps=w, **kw)
