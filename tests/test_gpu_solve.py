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


def canon(rec, n):
    """Records as (prefix, sorted remaining set, depth): equal up to the order
    in which a record lists its remaining jobs."""
    out = []
    for r in rec:
        d = int(r[n])
        out.append((tuple(r[:d]), tuple(sorted(r[d:n])), d))
    return out


def frontier_20x20(count):
    n = 20
    p, ub_perm, rec = inputs.pool_workload(n, 20, 1, count)
    return p, ub_perm, rec[rec[:, n] <= n - 2]


@pytest.mark.parametrize("pool,iters", [(4096, 3), (2**15, 1), (100, 7)])
def test_start_from_frontier_matches_oracle(F, pool, iters):
    """The bench step: a frontier of random 20 x 20 prefixes as the starting
    stack, UB = makespan of a random permutation, a few iterations."""
    import torch
    n = 20
    p, ub_perm, rec = frontier_20x20(40000)
    ub = oracle.makespan(p, ub_perm)
    ref = oracle.solve(p, ub0=ub, pool=pool, init_nodes=rec, max_iterations=iters, trace_cap=16,
                       export_stack=True)
    inst = F.fsp_create_instance(p)
    for init in (rec, torch.from_numpy(rec).cuda()):
        out = np.zeros((len(rec) + pool * iters, 32), np.uint8)
        got = F.fsp_solve(inst, ub0=ub, pool_size=pool, init_nodes=init, max_iterations=iters,
                          trace_cap=16, out_nodes=out, profile=True)
        same(got, ref)
        assert got["stack_left"] == ref["stack_left"]
        assert canon(out[: got["stack_left"]], n) == canon(ref["stack"], n)
        assert got["bound_ms"] > 0 and got["select_ms"] > 0 and got["compact_ms"] > 0


@pytest.mark.parametrize("pool,cut", [(1, 5), (16, 3), (256, 2)])
def test_resume_on_gpu(F, pool, cut):
    p = inputs.instance(9, 4, 151)
    inst = F.fsp_create_instance(p)
    full = F.fsp_solve(inst, pool_size=pool)
    out = np.zeros((4096, 16), np.uint8)
    a = F.fsp_solve(inst, pool_size=pool, max_iterations=cut, out_nodes=out)
    assert a["status"] == F.INCOMPLETE and a["iterations"] == cut
    b = F.fsp_solve(inst, ub0=a["cmax"], ub0_perm=a["perm"], pool_size=pool,
                    init_nodes=out[: a["stack_left"]])
    assert b["cmax"] == full["cmax"] == oracle.bruteforce(p)[0]
    for k in ("nodes_bounded", "nodes_branched", "nodes_pruned", "leaves", "iterations"):
        assert a[k] + b[k] == full[k], k
    assert list(b["perm"]) == list(full["perm"])


def test_init_nodes_validated_on_gpu(F):
    p = inputs.instance(6, 3, 161)
    inst = F.fsp_create_instance(p)
    rec = np.zeros((2, 16), np.uint8)
    rec[:, :6] = [0, 1, 2, 3, 4, 5]
    rec[:, 6] = 2
    rec[1, 6] = 5  # depth n-1
    with pytest.raises(F.FspError) as e:
        F.fsp_solve(inst, init_nodes=rec)
    assert e.value.code == F.ERR_ARG
    got = F.fsp_solve(inst, init_nodes=rec[:1])
    ref = oracle.solve(p, init_nodes=rec[:1])
    assert got["cmax"] == ref["cmax"] and got["nodes_bounded"] == ref["bounded"]


@pytest.mark.parametrize("n,m,seed,pool", [(12, 5, 0, 1024), (9, 20, 88, 64), (10, 10, 87, 7)])
def test_v1_search_kernels_match_oracle(F, n, m, seed, pool, monkeypatch):
    monkeypatch.setenv("FSP_BOUND_V1", "1")
    p = inputs.instance(n, m, seed)
    ref = oracle.solve(p, pool=pool, trace_cap=100000)
    got = F.fsp_solve(F.fsp_create_instance(p), pool_size=pool, trace_cap=100000)
    same(got, ref)


def test_wide_start_records_match_oracle(F):
    """Start records of n >= 64 jobs (their own validation kernel): a few
    iterations from random prefixes equal the oracle's; a malformed one is
    rejected."""
    import torch
    n, m = 70, 5
    p = inputs.instance(n, m, 171)
    rec = inputs.random_prefix_pool(n, 300, inputs.SplitMix64(172))
    rec[:, n] = np.minimum(rec[:, n], n - 2)
    ub = oracle.makespan(p, list(range(n)))
    inst = F.fsp_create_instance(p)
    ref = oracle.solve(p, ub0=ub, pool=512, init_nodes=rec, max_iterations=3, trace_cap=8)
    for init in (rec, torch.from_numpy(rec).cuda()):
        got = F.fsp_solve(inst, ub0=ub, pool_size=512, init_nodes=init, max_iterations=3, trace_cap=8)
        same(got, ref)
    bad = rec.copy()
    bad[5, 0] = bad[5, 1]
    with pytest.raises(F.FspError) as e:
        F.fsp_solve(inst, ub0=ub, pool_size=512, init_nodes=bad, max_iterations=3)
    assert e.value.code == F.ERR_ARG


def test_device_start_records_in_place_or_copied(F):
    """Start records on the device or in pinned host memory are read in place
    when 16-byte aligned and copied first otherwise: every path gives the
    pageable host records' search, and a malformed record is rejected."""
    import torch
    p, ub_perm, rec = frontier_20x20(3000)
    ub = oracle.makespan(p, ub_perm)
    ref = oracle.solve(p, ub0=ub, pool=2048, init_nodes=rec, max_iterations=2, trace_cap=4)
    inst = F.fsp_create_instance(p)
    flat = torch.zeros(rec.size + 8, dtype=torch.uint8, device="cuda")
    flat[8:] = torch.from_numpy(rec.reshape(-1)).cuda()
    odd = flat[8:].view(rec.shape)  # 8 bytes past an aligned base: copied first
    assert odd.data_ptr() % 16 == 8
    bad = rec.copy()
    bad[77, 3] = bad[77, 4]
    cases = ((torch.from_numpy(rec).cuda(), torch.from_numpy(bad).cuda()),
             (torch.from_numpy(rec).pin_memory(), torch.from_numpy(bad).pin_memory()), (odd, None))
    for init, wrong in cases:
        got = F.fsp_solve(inst, ub0=ub, pool_size=2048, init_nodes=init, max_iterations=2, trace_cap=4)
        same(got, ref)
        if wrong is not None:
            with pytest.raises(F.FspError) as e:
                F.fsp_solve(inst, ub0=ub, pool_size=2048, init_nodes=wrong, max_iterations=2)
            assert e.value.code == F.ERR_ARG


def test_large_start_stack_matches_oracle(F):
    """More than 2048 blocks of 256 start records: the running children counts
    come from the single-CTA scan of the block sums.  Two iterations equal the
    oracle's, and a malformed record far down the stack is rejected."""
    import torch
    p, ub_perm, rec = frontier_20x20(700000)
    assert len(rec) > 2048 * 256
    ub = oracle.makespan(p, ub_perm)
    ref = oracle.solve(p, ub0=ub, pool=8192, init_nodes=rec, max_iterations=2, trace_cap=4)
    inst = F.fsp_create_instance(p)
    got = F.fsp_solve(inst, ub0=ub, pool_size=8192, init_nodes=torch.from_numpy(rec).cuda(), max_iterations=2,
                      trace_cap=4)
    same(got, ref)
    assert got["iterations"] == 2 and got["time_ms"] > 0  # launched ahead, none past the cap
    bad = rec.copy()
    bad[600001, 0] = 20
    with pytest.raises(F.FspError) as e:
        F.fsp_solve(inst, ub0=ub, pool_size=8192, init_nodes=bad, max_iterations=2)
    assert e.value.code == F.ERR_ARG


def test_bench_step_matches_oracle(F):
    """The benchmark step at its full size, in the configuration bench.py
    times: one iteration with a pool of 2^18 children from the 248,115-record
    20 x 20 seed-1 frontier held on the device (read in place), UB = makespan
    of the seed's random permutation, phase timing on.  Counters, UB,
    incumbent and the whole stack left equal the oracle's."""
    import torch
    n, pool = 20, 2**18
    p, ub_perm, rec = frontier_20x20(2**18)
    ub = oracle.makespan(p, ub_perm)
    ref = oracle.solve(p, ub0=ub, pool=pool, init_nodes=rec, max_iterations=1, trace_cap=1, export_stack=True)
    inst = F.fsp_create_instance(p)
    out = torch.zeros((len(rec) + pool, inst.stride), dtype=torch.uint8, device="cuda")
    got = F.fsp_solve(inst, ub0=ub, pool_size=pool, init_nodes=torch.from_numpy(rec).cuda(), max_iterations=1,
                      trace_cap=1, out_nodes=out, profile=True)
    same(got, ref)
    k = got["stack_left"]
    assert k == ref["stack_left"]
    assert canon(out[:k].cpu().numpy(), n) == canon(ref["stack"], n)


@pytest.mark.parametrize("pdl", ["0", "1"])
def test_bench_step_and_search_in_both_launch_orders(F, pdl, monkeypatch):
    """The step kernels launched with programmatic stream serialization (the
    default: a kernel may start while the one ahead finishes and waits for
    its results in place) or in plain stream order (FSP_PDL=0): the bench
    step as bench.py times it (no phase events) equals the oracle's, stack
    included, and a 20 x 20 search of many iterations launched ahead gives
    the same trace and stack either way."""
    import torch
    monkeypatch.setenv("FSP_PDL", pdl)
    n, pool = 20, 2**18
    p, ub_perm, rec = frontier_20x20(2**18)
    ub = oracle.makespan(p, ub_perm)
    ref = oracle.solve(p, ub0=ub, pool=pool, init_nodes=rec, max_iterations=1, trace_cap=1, export_stack=True)
    inst = F.fsp_create_instance(p)
    out = torch.zeros((len(rec) + pool, inst.stride), dtype=torch.uint8, device="cuda")
    got = F.fsp_solve(inst, ub0=ub, pool_size=pool, init_nodes=torch.from_numpy(rec).cuda(), max_iterations=1,
                      trace_cap=1, out_nodes=out)
    same(got, ref)
    k = got["stack_left"]
    assert canon(out[:k].cpu().numpy(), n) == canon(ref["stack"], n)
    q = inputs.instance(20, 20, 6)
    qi = F.fsp_create_instance(q)
    u, perm = F.fsp_neh(qi)
    a = F.fsp_solve(qi, ub0=u, ub0_perm=perm, pool_size=8192, node_budget=3_000_000, trace_cap=4096)
    monkeypatch.setenv("FSP_PDL", "1" if pdl == "0" else "0")
    b = F.fsp_solve(qi, ub0=u, ub0_perm=perm, pool_size=8192, node_budget=3_000_000, trace_cap=4096)
    for key in ("status", "cmax", "nodes_bounded", "nodes_branched", "nodes_pruned", "leaves", "iterations",
                "incumbent_updates", "stack_left"):
        assert a[key] == b[key], key
    assert np.array_equal(a["trace"], b["trace"])
