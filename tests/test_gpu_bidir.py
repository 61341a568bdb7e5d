"""GPU parity of bidirectional branching with the oracle (oracle.bound_pool2,
oracle.solve_bidir): the bound of bidirectional records on the packed kernel
and on the generic one, across shapes, ragged pools and the edge splits (no
suffix, nothing left, no prefix); malformed records; and whole searches with
every counter, the trace, the optimum and the permutation."""
import numpy as np
import pytest

import oracle
from paper_1206_4973_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_1206_4973_gb300 import build, fsp
    build.build()
    fsp.load()
    assert torch.cuda.is_available()
    return fsp


def bidir_pool(n, count, seed, stride):
    rng = np.random.default_rng(seed)
    rec = np.zeros((count, stride), np.uint8)
    for t in range(count):
        rec[t, :n] = rng.permutation(n)
        d1 = int(rng.integers(0, n + 1))
        d2 = int(rng.integers(0, n - d1 + 1))
        if t % 7 == 0:
            d2 = 0                      # a forward node
        elif t % 11 == 0:
            d2 = n - d1                 # nothing left: the makespan
        elif t % 13 == 0:
            d1, d2 = 0, min(d2, n)      # no prefix
        rec[t, n], rec[t, n + 1] = d1, d2
    return rec


# packed kernel: n <= 31, m in {5, 10, 20} (records of 16, 32 and 48 bytes);
# generic kernel: the rest
SHAPES = [(20, 20, 1), (12, 5, 0), (13, 10, 3), (15, 20, 4), (30, 10, 5), (31, 20, 6), (29, 5, 7),
          (50, 20, 8), (9, 3, 9), (40, 7, 10), (2, 5, 11)]


@pytest.mark.parametrize("n,m,seed", SHAPES)
def test_bidir_bounds_match_oracle(F, n, m, seed, monkeypatch):
    import torch
    p = inputs.instance(n, m, seed)
    stride = F.fsp_node_stride_bidir(n)
    assert stride == oracle.stride2(n)
    rec = bidir_pool(n, 1537, seed + 300, stride)
    want = oracle.bound_pool2(p, rec)
    inst = F.fsp_create_instance(p)
    nodes = torch.from_numpy(rec).cuda()
    got = F.fsp_bound_pool_bidir(inst, nodes).cpu().numpy()
    F.fsp_check_status(inst)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    monkeypatch.setenv("FSP_BOUND_V1", "1")  # the generic kernel on every shape
    got = F.fsp_bound_pool_bidir(inst, nodes).cpu().numpy()
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


def test_bidir_with_no_suffix_is_the_forward_bound(F):
    import torch
    n, m = 20, 20
    p, _, rec = inputs.pool_workload(n, m, 1, 2000)
    rec2 = np.zeros((len(rec), F.fsp_node_stride_bidir(n)), np.uint8)
    rec2[:, :n + 1] = rec[:, :n + 1]
    inst = F.fsp_create_instance(p)
    a = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    b = F.fsp_bound_pool_bidir(inst, torch.from_numpy(rec2).cuda()).cpu().numpy()
    assert np.array_equal(a, b)


def test_bidir_malformed_records_are_flagged(F):
    import torch
    n, m = 12, 5
    p = inputs.instance(n, m, 3)
    stride = F.fsp_node_stride_bidir(n)
    rec = bidir_pool(n, 64, 5, stride)
    rec[3, 0] = rec[3, 1]             # repeated job
    rec[9, n], rec[9, n + 1] = 8, 5   # d1 + d2 > n
    rec[20, 2] = n                    # job id out of range
    inst = F.fsp_create_instance(p)
    got = F.fsp_bound_pool_bidir(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    assert got[3] == F.LB_INVALID and got[9] == F.LB_INVALID and got[20] == F.LB_INVALID
    good = np.ones(64, bool)
    good[[3, 9, 20]] = False
    assert np.array_equal(got[good], oracle.bound_pool2(p, rec[good]))
    with pytest.raises(F.FspError):
        F.fsp_check_status(inst)


# GPU counter -> oracle counter
KEYS = {"nodes_bounded": "bounded", "nodes_branched": "branched", "nodes_pruned": "pruned", "leaves": "leaves",
        "iterations": "iterations", "incumbent_updates": "incumbent_updates"}


@pytest.mark.parametrize("family", [True, False])
@pytest.mark.parametrize("n,m,seed,pool", [(12, 5, 0, 1024), (10, 4, 21, 1), (10, 4, 21, 7), (11, 20, 22, 300),
                                           (14, 10, 23, 4096), (9, 3, 24, 64), (16, 5, 25, 20000),
                                           (15, 10, 26, 500), (13, 20, 27, 3000), (17, 5, 28, 2)])
def test_bidir_search_matches_oracle(F, n, m, seed, pool, family, monkeypatch):
    """Whole searches, on the family kernel (children of a parent bounded
    together, both directions) and on the per-child kernels (FSP_FAMILY=0)."""
    if not family:
        monkeypatch.setenv("FSP_FAMILY", "0")
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst, pool_size=pool, trace_cap=100000, branching=F.BRANCH_BIDIR)
    want = oracle.solve_bidir(p, pool=pool, trace_cap=100000)
    assert got["status"] == F.OK and want["status"] == oracle.OK
    assert got["cmax"] == want["cmax"]
    for k, ko in KEYS.items():
        assert got[k] == want[ko], k
    assert np.array_equal(got["trace"], want["trace"])
    assert list(got["perm"]) == list(want["perm"])


@pytest.mark.parametrize("n,m,seed", [(8, 4, 31), (9, 5, 32), (7, 20, 33)])
def test_bidir_search_reaches_the_optimum(F, n, m, seed):
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    best, _ = oracle.bruteforce(p)
    for pool in (1, 50, 5000):
        r = F.fsp_solve(inst, pool_size=pool, branching=F.BRANCH_BIDIR)
        assert r["cmax"] == best
        assert oracle.makespan(p, r["perm"]) == best


def test_bidir_budget_and_tuned_pool(F):
    """A node budget stops the bidirectional search like the forward one; the
    tuned pool's schedule replays on the oracle... (the oracle has no schedule
    input for this search, so the tuned run is checked for its optimum)."""
    p = inputs.instance(15, 5, 40)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst, pool_size=512, node_budget=20000, branching=F.BRANCH_BIDIR)
    want = oracle.solve_bidir(p, pool=512, node_budget=20000)
    assert got["status"] == F.INCOMPLETE and want["status"] == oracle.INCOMPLETE
    for k, ko in KEYS.items():
        assert got[k] == want[ko], k
    assert got["cmax"] == want["cmax"]
    full = F.fsp_solve(inst, pool_size=0, branching=F.BRANCH_BIDIR)
    assert full["cmax"] == oracle.solve(p, pool=4096)["cmax"]


def test_bidir_rejects_start_records(F):
    p = inputs.instance(8, 3, 1)
    inst = F.fsp_create_instance(p)
    rec = np.zeros((1, inst.stride), np.uint8)
    rec[0, :8] = np.arange(8)
    with pytest.raises(F.FspError):
        F.fsp_solve(inst, init_nodes=rec, branching=F.BRANCH_BIDIR)


def test_bidir_family_on_the_20x20_frontier_matches_oracle(F):
    """Bidirectional records with prefixes and suffixes of every length as
    start records are not accepted; instead a budgeted 20 x 20 search runs a
    few thousand iterations of both directions against the oracle."""
    p = inputs.instance(20, 20, 1)
    inst = F.fsp_create_instance(p)
    ub = oracle.neh(p)[0]
    got = F.fsp_solve(inst, ub0=ub, pool_size=2048, node_budget=300000, trace_cap=100000,
                      branching=F.BRANCH_BIDIR)
    want = oracle.solve_bidir(p, ub0=ub, pool=2048, node_budget=300000, trace_cap=100000)
    for k, ko in KEYS.items():
        assert got[k] == want[ko], k
    assert got["cmax"] == want["cmax"]
    assert np.array_equal(got["trace"], want["trace"])
