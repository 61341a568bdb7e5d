"""The batched solver (one persistent launch, device work queue, CUDA graph)
against the oracle: every instance's search equals oracle.solve with the
same pool, the NEH UB and the same node budget, bit-exact."""
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


def check(F, instances, res, pools, budgets, ub0=None):
    for i, (p, r) in enumerate(zip(instances, res)):
        if ub0 is None:
            u, perm0 = oracle.neh(p)
        else:
            u, perm0 = int(ub0[i]), None
        ref = oracle.solve(p, ub0=u, pool=int(pools[i]), node_budget=int(budgets[i]), ub0_perm=perm0)
        assert r["status"] == ref["status"], i
        assert r["cmax"] == ref["cmax"], i
        for k in ("bounded", "branched", "pruned", "leaves", "iterations", "incumbent_updates"):
            key = "nodes_" + k if k in ("bounded", "branched", "pruned") else k
            assert r[key] == ref[k], (i, k)
        if ref["perm"] is not None:
            assert list(r["perm"]) == list(ref["perm"]), i


def test_mixed_batch_matches_oracle(F):
    shapes = inputs.batch_shapes(24, first_seed=100)
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    pools = np.array([(64, 256, 1024)[i % 3] for i in range(24)], np.int64)
    budgets = np.full(24, 20000, np.int64)
    B = F.Batch(instances, pools, budgets)
    B.run()
    res = B.results()
    check(F, instances, res, pools, budgets)
    B.run()  # the graph replays: same results
    again = B.results()
    for a, b in zip(again, res):
        assert {k: v for k, v in a.items() if k != "perm"} == {k: v for k, v in b.items() if k != "perm"}
        assert list(a["perm"]) == list(b["perm"])


def test_small_instances_solved_to_optimality(F):
    shapes = [(9, 5, 1), (10, 10, 2), (16, 20, 3), (12, 5, 4), (7, 5, 5), (11, 10, 6), (2, 5, 7), (3, 10, 8)]
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    pools = np.array([32, 512, 100, 1, 7, 2048, 4, 16], np.int64)
    budgets = np.array([0, 0, 30000, 0, 0, 0, 0, 0], np.int64)
    B = F.Batch(instances, pools, budgets)
    B.run()
    res = B.results()
    check(F, instances, res, pools, budgets)
    for p, r in zip(instances, res):
        if p.shape[0] <= 9:
            assert r["cmax"] == oracle.bruteforce(p)[0] and r["status"] == F.OK


def test_given_upper_bounds(F):
    instances = [inputs.instance(10, 5, 31), inputs.instance(12, 10, 32)]
    ub0 = np.array([oracle.neh(p)[0] + 5 for p in instances], np.int32)
    pools, budgets = np.array([128, 64], np.int64), np.array([0, 5000], np.int64)
    B = F.Batch(instances, pools, budgets, ub0=ub0)
    B.run()
    check(F, instances, B.results(), pools, budgets, ub0=ub0)


def test_rejects_unsupported_shapes(F):
    with pytest.raises(F.FspError):
        F.Batch([inputs.instance(10, 7, 1)], [64])
    with pytest.raises(F.FspError):
        F.Batch([inputs.instance(40, 5, 1)], [64])
    with pytest.raises(F.FspError):
        F.Batch([inputs.instance(10, 5, 1)], [5000])


def test_pool_tuning_per_shape(F):
    shapes = inputs.batch_shapes(16, first_seed=100)
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    pools = F.fsp_batch_tune_pools(instances, probe_budget=20000)
    assert set(pools.tolist()) <= {128, 256, 512, 1024, 2048, 4096}
    for i in range(16):
        for j in range(16):
            if shapes[i][:2] == shapes[j][:2]:
                assert pools[i] == pools[j]


def test_split_mode_reaches_the_same_optima(F):
    """Split mode (the roots' subtrees as work items, a shared UB per
    instance): every instance solved to optimality gives the oracle's
    optimum and a schedule attaining it; counters are totals over the
    subtrees (another exploration order), so only their consistency is
    checked."""
    shapes = [(9, 5, 1), (10, 10, 2), (12, 5, 4), (7, 5, 5), (11, 10, 6), (2, 5, 7), (3, 10, 8), (12, 5, 9),
              (10, 5, 10), (9, 10, 11)] + list(inputs.batch_shapes(12, first_seed=100)[:8])
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    k = len(instances)
    pools = np.array([(64, 256, 1024, 7)[i % 4] for i in range(k)], np.int64)
    budgets = np.zeros(k, np.int64)
    budgets[-8:] = 400000  # the 20- and 50-job shapes: capped, checked for consistency only
    whole = F.Batch(instances, pools, budgets)
    whole.run()
    ref = whole.results()
    B = F.Batch(instances, pools, budgets, split=True)
    for _ in range(2):  # the graph replays from scratch
        B.run()
        res = B.results()
        for i, (p, r, w) in enumerate(zip(instances, res, ref)):
            assert r["status"] in (F.OK, F.INCOMPLETE), i
            assert oracle.makespan(p, r["perm"]) == r["cmax"], i
            assert r["nodes_bounded"] >= r["nodes_pruned"] + r["leaves"], i  # the rest survived
            if r["status"] == F.OK and p.shape[0] <= 12:  # small enough for the serial oracle
                best = oracle.solve(p, pool=4096)["cmax"] if p.shape[0] > 9 else oracle.bruteforce(p)[0]
                assert r["cmax"] == best, i
            if r["status"] == F.OK and w["status"] == F.OK:  # the whole-instance search equals the oracle's
                assert r["cmax"] == w["cmax"], i
            if budgets[i] == 0:
                assert r["status"] == F.OK, i
    B.set_split(False)  # back to whole instances: the bit-exact search
    B.run()
    check(F, instances, B.results(), pools, budgets)


def test_bidirectional_batch_matches_oracle(F):
    """Bidirectional branching in the batch: each instance's search equals
    oracle.solve_bidir with the same pool, NEH UB and node budget (every
    counter, the optimum); split mode reaches the same optima."""
    shapes = list(inputs.batch_shapes(16, first_seed=200)) + [(9, 5, 1), (12, 10, 2), (2, 5, 3), (14, 5, 4)]
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    k = len(instances)
    pools = np.array([(64, 256, 1024, 3)[i % 4] for i in range(k)], np.int64)
    budgets = np.array([20000] * 16 + [0] * 4, np.int64)
    B = F.Batch(instances, pools, budgets)
    B.set_bidir(True)
    B.run()
    res = B.results()
    for i, (p, r) in enumerate(zip(instances, res)):
        u, _ = oracle.neh(p)
        ref = oracle.solve_bidir(p, ub0=u, pool=int(pools[i]), node_budget=int(budgets[i]))
        assert r["status"] == ref["status"], i
        assert r["cmax"] == ref["cmax"], i
        for key in ("bounded", "branched", "pruned", "leaves", "iterations", "incumbent_updates"):
            name = "nodes_" + key if key in ("bounded", "branched", "pruned") else key
            assert r[name] == ref[key], (i, key)
        assert oracle.makespan(p, r["perm"]) == r["cmax"], i
    B.set_split(True)
    B.run()
    for i, (a, b) in enumerate(zip(res, B.results())):
        assert oracle.makespan(instances[i], b["perm"]) == b["cmax"], i
        if a["status"] == F.OK and b["status"] == F.OK:
            assert a["cmax"] == b["cmax"], i
    with pytest.raises(F.FspError):  # records of 32 jobs + 2 bytes: no bidirectional batch kernel
        F.Batch([inputs.instance(31, 20, 1)], [64]).set_bidir(True)


def test_block_shapes_per_instance_give_the_same_searches(F):
    """Every instance with its own block shape (1 to 20 warps per CTA, the
    instances of one shape split over several block shapes, so several
    launches run side by side): the whole-instance searches are the oracle's,
    counter for counter, as with the default 8 warps; split mode reaches the
    same optima with every block shape."""
    shapes = inputs.batch_shapes(24, first_seed=300)
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    pools = np.array([(64, 256, 1024)[i % 3] for i in range(24)], np.int64)
    budgets = np.full(24, 20000, np.int64)
    # 16 warps of 50 x 10 tables exceed a CTA's shared memory: at most 12 there
    warps = np.array([min((1, 2, 4, 8, 12, 16, 20)[i % 7], 12 if shapes[i][:2] == (50, 10) else 20)
                      for i in range(24)], np.int32)
    B = F.Batch(instances, pools, budgets, warps=warps)
    B.run()
    res = B.results()
    check(F, instances, res, pools, budgets)
    B.set_warps(None)  # back to 8 warps for all: the same results
    B.run()
    for a, b in zip(B.results(), res):
        assert {k: v for k, v in a.items() if k != "perm"} == {k: v for k, v in b.items() if k != "perm"}
        assert list(a["perm"]) == list(b["perm"])
    small = [inputs.instance(n, m, s) for n, m, s in [(9, 5, 1), (10, 10, 2), (12, 5, 4), (11, 10, 6), (13, 5, 9)]]
    sp = np.array([256, 512, 64, 2048, 128], np.int64)
    S = F.Batch(small, sp, split=True, warps=np.array([4, 16, 2, 8, 12], np.int32))
    S.run()
    for p, r in zip(small, S.results()):
        assert r["status"] == F.OK and r["cmax"] == oracle.solve(p, ub0=oracle.neh(p)[0], pool=1024)["cmax"]
        assert oracle.makespan(p, r["perm"]) == r["cmax"]
    S.set_bidir(True)
    S.run()
    for p, r in zip(small, S.results()):
        assert r["status"] == F.OK and oracle.makespan(p, r["perm"]) == r["cmax"]


def test_block_shape_rejected_when_it_does_not_fit(F):
    B = F.Batch([inputs.instance(12, 5, 1), inputs.instance(50, 10, 2)], [64, 64], budgets=[20000, 20000])
    with pytest.raises(F.FspError):
        B.set_warps(np.array([8, 21], np.int32))  # more than 20 warps
    with pytest.raises(F.FspError):
        B.set_warps(np.array([8, 16], np.int32))  # 50 x 10 tables of 16 warps exceed a CTA's shared memory
    B.run()  # unchanged and still usable
    assert all(r["status"] in (F.OK, F.INCOMPLETE) for r in B.results())


def test_block_shape_tuning_per_shape(F):
    shapes = inputs.batch_shapes(16, first_seed=100)
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    pools = np.full(16, 512, np.int64)
    w = F.fsp_batch_tune_warps(instances, pools, probe_budget=5000)
    assert set(w.tolist()) <= {4, 8, 12, 16, 20}
    for i in range(16):
        for j in range(16):
            if shapes[i][:2] == shapes[j][:2]:
                assert w[i] == w[j]


def test_class_stats_describe_the_last_launch(F):
    """fsp_batch_class_stats: one entry per (shape, warps) class, the CTAs of
    its launch and their lifetimes from the global timer, consistent with one
    another and with the launch span; split mode lists the subtrees as items."""
    shapes = [(12, 5, 1), (12, 5, 2), (15, 10, 3), (15, 10, 4), (20, 5, 5)]
    instances = [inputs.instance(n, m, s) for n, m, s in shapes]
    B = F.Batch(instances, np.full(5, 256, np.int64), np.full(5, 20000, np.int64),
                warps=np.array([8, 8, 4, 16, 8], np.int32))
    B.run()
    B.results()
    st = B.class_stats()
    assert sorted((c["n"], c["m"], c["warps"]) for c in st) == [(12, 5, 8), (15, 10, 4), (15, 10, 16), (20, 5, 8)]
    for c in st:
        assert 1 <= c["ctas"] <= c["items"] == c["instances"]
        assert 0.0 <= c["busy_min_ms"] <= c["busy_mean_ms"] <= c["busy_max_ms"] <= c["launch_span_ms"] + 1e-6
        assert c["first_start_ms"] <= c["last_end_ms"] <= c["launch_span_ms"] + 1e-6
    B.set_split(True)
    B.run()
    B.results()
    st = B.class_stats()
    for c in st:
        assert c["items"] == c["instances"] * c["n"]
        assert 1 <= c["ctas"] <= c["items"]
        assert c["donated"] >= 0


def test_donated_nodes_keep_the_optima(F):
    """Split mode with one hard instance among easy ones: once the item queue
    is empty the CTAs still searching hand nodes to the waiting ones; the
    optima stay the oracle's (whole-instance batch and oracle.solve), every
    returned schedule attains its makespan, and nodes were donated."""
    hard = inputs.instance(15, 10, 101)
    easy = [inputs.instance(9, 5, s) for s in range(8)]
    instances = [hard] + easy
    pools = np.full(len(instances), 512, np.int64)
    whole = F.Batch(instances, pools)
    whole.run()
    ref = whole.results()
    for bidir in (False, True):
        S = F.Batch(instances, pools, split=True)
        if bidir:
            S.set_bidir(True)
        S.run()
        got = S.results()
        for p, a, b in zip(instances, got, ref):
            assert a["status"] == F.OK and a["cmax"] == b["cmax"]
            assert oracle.makespan(p, a["perm"]) == a["cmax"]
        assert sum(c["donated"] for c in S.class_stats()) > 0
    for p, r in zip(easy, ref[1:]):
        assert r["cmax"] == oracle.bruteforce(p)[0]


def test_split_wait_limit_reports_timeout_and_recovers(F):
    """The wait limit of split mode's donations, made to run out on the host's
    side (fsp_batch_set_test_hold: each launch starts with the donation lock
    taken and a donated node marked waiting, and nothing releases them).  Every
    wait ends after 1 s, the kernel returns, and every instance reports
    FSP_ERR_TIMEOUT; with the hook off, the same batch on the same context then
    returns the optima of brute force."""
    import time
    instances = [inputs.instance(7, 5, s) for s in range(3)]
    pools = np.full(len(instances), 256, np.int64)
    S = F.Batch(instances, pools, split=True)
    S.set_test_hold(True)
    t0 = time.perf_counter()
    S.run()
    got = S.results()
    assert time.perf_counter() - t0 < 30
    assert [r["status"] for r in got] == [F.ERR_TIMEOUT] * len(instances)
    S.set_test_hold(False)
    S.run()
    got = S.results()
    for p, r in zip(instances, got):
        assert r["status"] == F.OK and r["cmax"] == oracle.bruteforce(p)[0]
        assert oracle.makespan(p, r["perm"]) == r["cmax"]
    S.close()
