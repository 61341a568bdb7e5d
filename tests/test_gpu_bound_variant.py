"""The heads bound variant (release times raised by the smallest heads) on every
GPU path: per-node kernels (register and generic shapes), the family kernel,
the per-child search kernels and the learned order all give the oracle's
bounds and searches bit for bit."""
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


# register kernels (m in {5,10,20}, n <= 63) and the generic ones (other m, n > 63)
@pytest.mark.parametrize("n,m,seed", [(20, 20, 1), (12, 5, 2), (33, 10, 3), (100, 20, 4), (30, 7, 5), (70, 3, 6)])
def test_bound_pool_heads_matches_oracle(F, n, m, seed):
    import torch
    p = inputs.instance(n, m, seed)
    rec = inputs.random_prefix_pool(n, 3000, inputs.SplitMix64(seed + 50))
    rec[::7, n] = n - 1
    rec[::11, n] = n
    inst = F.fsp_create_instance(p)
    inst.set_bound(F.BOUND_HEADS)
    got = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    F.fsp_check_status(inst)
    assert np.array_equal(got, oracle.bound_pool(p, rec, bound=1))
    inst.set_bound(F.BOUND_BASE)
    base = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    assert np.array_equal(base, oracle.bound_pool(p, rec))
    assert np.all(got >= base)


@pytest.mark.parametrize("n,m,seed,pool", [(12, 5, 0, 1024), (9, 7, 3, 64), (10, 20, 8, 256), (11, 10, 9, 1)])
def test_solve_heads_matches_oracle(F, n, m, seed, pool):
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    inst.set_bound(F.BOUND_HEADS)
    r = F.fsp_solve(inst, pool_size=pool, trace_cap=100000)
    ref = oracle.solve(p, pool=pool, trace_cap=100000, bound=1)
    assert r["status"] == ref["status"] and r["cmax"] == ref["cmax"]
    for k in ("nodes_bounded", "nodes_branched", "nodes_pruned", "leaves", "iterations", "incumbent_updates"):
        assert r[k] == ref[{"nodes_bounded": "bounded", "nodes_branched": "branched", "nodes_pruned": "pruned",
                            "incumbent_updates": "incumbent_updates"}.get(k, k)], k
    assert np.array_equal(r["trace"], ref["trace"])
    assert list(r["perm"]) == list(ref["perm"])


@pytest.mark.parametrize("n,m,seed,pool", [(20, 20, 6, 8192), (50, 10, 7, 4096), (15, 5, 3, 512)])
def test_heads_children_bounds_and_kernels_agree(F, n, m, seed, pool):
    """Logged child bounds equal the oracle's; the family kernel, the per-child
    kernel and the learned order run the same search."""
    import torch
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    inst.set_bound(F.BOUND_HEADS)
    ub0, perm0 = F.fsp_neh(inst)
    kw = dict(ub0=ub0, ub0_perm=perm0, pool_size=pool, node_budget=60000, trace_cap=100000)
    cap = 40000
    log = torch.zeros((cap, inst.stride), dtype=torch.uint8, device="cuda")
    lbs = torch.zeros(cap, dtype=torch.int32, device="cuda")
    a = F.fsp_solve(inst, log_nodes=log, log_lbs=lbs, **kw)
    k = a["logged"]
    rec = log[:k].cpu().numpy()
    idx = np.unique(np.linspace(0, k - 1, min(k, 12000)).astype(np.int64))
    assert np.array_equal(lbs[:k].cpu().numpy()[idx], oracle.bound_pool(p, rec[idx], bound=1))
    os.environ["FSP_FAMILY"] = "0"
    try:
        b = F.fsp_solve(inst, **kw)
    finally:
        del os.environ["FSP_FAMILY"]
    mlp = F.Mlp(2 * m + 1, 128, m * (m - 1) // 2, seed=seed)
    c = F.fsp_solve(inst, model=mlp, topk=4, **kw)
    for key in KEYS:
        assert a[key] == b[key] == c[key], key
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["trace"], c["trace"])


def test_set_bound_rejects_unknown_variant(F):
    inst = F.fsp_create_instance(inputs.instance(6, 3, 1))
    with pytest.raises(F.FspError):
        inst.set_bound(7)
