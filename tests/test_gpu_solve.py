"""GPU parity of the device branch-and-bound with the CPU oracle: optimal
makespan, permutation, every counter and the per-iteration trace (parents,
children, survivors, UB) bit-exact, across pool sizes, shapes, budgets,
replayed pool schedules and the degenerate cases."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1206_4973_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_1206_4973_gb300 import build, fsp
    build.build()
    fsp.load()
    assert torch.cuda.is_available()
    return fsp


def same(gpu, ref, trace=True):
    assert gpu["status"] == ref["status"]
    assert gpu["cmax"] == ref["cmax"]
    assert gpu["nodes_bounded"] == ref["bounded"]
    assert gpu["nodes_branched"] == ref["branched"]
    assert gpu["nodes_pruned"] == ref["pruned"]
    assert gpu["leaves"] == ref["leaves"]
    assert gpu["iterations"] == ref["iterations"]
    assert gpu["incumbent_updates"] == ref["incumbent_updates"]
    if ref["perm"] is None:
        assert gpu["perm"] is None
    else:
        assert list(gpu["perm"]) == list(ref["perm"])
    if trace:
        assert np.array_equal(gpu["trace"], ref["trace"])


def test_config_12x5_seed0_pool1024(F):
    n, m = 12, 5
    p = inputs.instance(n, m, 0)
    ref = oracle.solve(p, pool=1024, trace_cap=100000)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst, pool_size=1024, trace_cap=100000)
    same(got, ref)
    g = json.load(open(os.path.join(GOLDEN, "solve_12x5_seed0.json")))
    assert got["cmax"] == g["cmax"] and list(got["perm"]) == g["perm"]
    assert got["nodes_bounded"] == g["bounded"]


@pytest.mark.parametrize("n,m,seed", [(2, 3, 80), (3, 2, 1), (5, 2, 81), (6, 3, 82), (7, 5, 83),
                                      (8, 4, 84), (9, 3, 86), (10, 10, 87), (9, 20, 88)])
@pytest.mark.parametrize("pool", [1, 3, 7, 64, 5000])
def test_small_solves_match_oracle(F, n, m, seed, pool):
    p = inputs.instance(n, m, seed)
    ref = oracle.solve(p, pool=pool, trace_cap=200000)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst, pool_size=pool, trace_cap=200000)
    same(got, ref)
    if n <= 9:
        assert got["cmax"] == oracle.bruteforce(p)[0]


def test_single_job(F):
    p = np.array([[4, 5, 6]], np.int32)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst)
    assert got["cmax"] == 15 and list(got["perm"]) == [0] and got["iterations"] == 0
    got = F.fsp_solve(inst, ub0=10)
    assert got["cmax"] == 10 and got["perm"] is None


def test_ub0_at_and_below_the_optimum(F):
    p = inputs.instance(8, 4, 111)
    opt, _ = oracle.bruteforce(p)
    inst = F.fsp_create_instance(p)
    for ub0 in (opt, opt - 1, opt + 1):
        ref = oracle.solve(p, ub0=ub0, pool=16, trace_cap=10000)
        got = F.fsp_solve(inst, ub0=ub0, pool_size=16, trace_cap=10000)
        same(got, ref)
    neh_c, neh_perm = oracle.neh(p)
    got = F.fsp_solve(inst, ub0=opt, ub0_perm=neh_perm, pool_size=16)
    assert got["cmax"] == opt and list(got["perm"]) == list(neh_perm)


@pytest.mark.parametrize("n,m,seed,budget,pool", [(20, 5, 2, 30000, 1024), (50, 10, 6, 20000, 4096),
                                                  (20, 20, 6, 50000, 8192), (100, 5, 4, 20000, 2048),
                                                  (15, 10, 9, 40000, 256)])
def test_budgeted_searches_match_oracle(F, n, m, seed, budget, pool):
    """Larger shapes, stopped by a node budget at the same iteration on both
    sides: every counter and the trace still agree exactly."""
    p = inputs.instance(n, m, seed)
    ub0, _ = oracle.neh(p)
    ref = oracle.solve(p, ub0=ub0, pool=pool, node_budget=budget, trace_cap=100000)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst, ub0=ub0, pool_size=pool, node_budget=budget, trace_cap=100000)
    same(got, ref)


def test_schedule_replay(F):
    p = inputs.instance(10, 5, 121)
    sched = [3, 50, 7, 1000, 2, 300]
    ref = oracle.solve(p, pool=1, schedule=sched, trace_cap=100000)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst, pool_size=1, schedule=sched, trace_cap=100000)
    same(got, ref)


def test_stack_capacity_error_keeps_state(F):
    p = inputs.instance(10, 5, 131)
    inst = F.fsp_create_instance(p)
    with pytest.raises(F.FspError) as e:
        F.fsp_solve(inst, pool_size=64, stack_capacity=40)
    assert e.value.code == F.ERR_CAPACITY
    # the instance is still usable afterwards
    ref = oracle.solve(p, pool=64)
    got = F.fsp_solve(inst, pool_size=64)
    assert got["cmax"] == ref["cmax"] and got["nodes_bounded"] == ref["bounded"]


def test_caller_workspace_and_stream(F):
    import torch
    p = inputs.instance(9, 5, 141)
    inst = F.fsp_create_instance(p)
    nbytes = F.fsp_solve_workspace_bytes(inst, pool_size=32)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    got = F.fsp_solve(inst, pool_size=32, workspace=ws, stream=s)
    ref = oracle.solve(p, pool=32)
    assert got["cmax"] == ref["cmax"] and got["nodes_bounded"] == ref["bounded"]
