"""The learned pair order changes which bounds are computed, never the search:
with any network and any K, the learned search cuts the same children,
explores the same nodes in the same order and finds the same incumbent as
the plain one (and as the oracle).  A trained network cuts more children by
their predicted pairs alone than an untrained one."""
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


def canon(rec, n):
    return [(tuple(r[: r[n]]), tuple(sorted(r[r[n]:n])), int(r[n])) for r in rec]


def run(F, inst, n, **kw):
    out = np.zeros((kw.get("pool_size", 1024) * 8 + 4096 * n, inst.stride), np.uint8)
    r = F.fsp_solve(inst, out_nodes=out, trace_cap=100000, **kw)
    r["stack"] = canon(out[: r["stack_left"]], n) if r["stack_left"] <= len(out) else None
    return r


def same(a, b):
    for k in KEYS:
        assert a[k] == b[k], k
    assert (a["perm"] is None) == (b["perm"] is None)
    if a["perm"] is not None:
        assert list(a["perm"]) == list(b["perm"])
    assert np.array_equal(a["trace"], b["trace"])
    assert a["stack"] == b["stack"]


@pytest.mark.parametrize("n,m,seed,pool,budget", [(12, 5, 0, 1024, 0), (10, 10, 87, 64, 0), (9, 20, 88, 64, 0),
                                                  (20, 20, 6, 8192, 60000), (50, 20, 7, 4096, 40000),
                                                  (33, 10, 21, 2048, 50000), (15, 7, 3, 256, 30000)])
def test_learned_order_gives_the_plain_search(F, n, m, seed, pool, budget):
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst) if budget else (F.UB_INF, None)
    kw = dict(ub0=ub0, ub0_perm=perm0, pool_size=pool, node_budget=budget)
    plain = run(F, inst, n, **kw)
    mlp = F.Mlp(2 * m + 1, 128, m * (m - 1) // 2, seed=seed)
    for topk in (1, 4, 8):
        learned = run(F, inst, n, model=mlp, topk=topk, **kw)
        same(learned, plain)
        assert learned["early_pruned"] <= learned["nodes_pruned"] + learned["leaves"]
    if budget == 0:
        ref = oracle.solve(p, pool=pool)
        assert plain["cmax"] == ref["cmax"] and plain["nodes_bounded"] == ref["bounded"]


def test_logging_stores_every_bounded_child(F):
    import torch
    n, m = 12, 5
    p = inputs.instance(n, m, 0)
    inst = F.fsp_create_instance(p)
    log = torch.zeros((5000, inst.stride), dtype=torch.uint8, device="cuda")
    r = F.fsp_solve(inst, pool_size=1024, log_nodes=log)
    assert r["logged"] == min(5000, r["nodes_bounded"])
    rec = log.cpu().numpy()
    # the first iteration bounds the root's children, by increasing job index
    for j in range(n):
        assert rec[j, 0] == j and rec[j, n] == 1
        assert list(rec[j, 1:n]) == [x for x in range(n) if x != j]
    got = F.fsp_bound_pool(inst, log).cpu().numpy()
    F.fsp_check_status(inst)
    assert np.array_equal(got[:2000], oracle.bound_pool(p, rec[:2000]))


def test_trained_network_cuts_more_than_untrained(F):
    """Train on children a plain 20 x 20 search logs, then compare the
    children cut by the top-4 predicted pairs with an untrained network."""
    import torch
    n, m = 20, 20
    P = m * (m - 1) // 2
    p = inputs.instance(n, m, 6)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst)
    log = torch.zeros((200000, inst.stride), dtype=torch.uint8, device="cuda")
    F.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=8192, node_budget=200000, log_nodes=log)
    x, y = F.fsp_node_features(inst, log)
    trained = F.Mlp(2 * m + 1, 128, P, seed=2)
    for it in range(400):
        s = (it * 4096) % (len(y) - 4096)
        trained.train_step(x[s:s + 4096], y[s:s + 4096], lr=2e-3)
    untrained = F.Mlp(2 * m + 1, 128, P, seed=2)
    kw = dict(ub0=ub0, ub0_perm=perm0, pool_size=8192, node_budget=300000)
    a = F.fsp_solve(inst, model=trained, topk=4, **kw)
    b = F.fsp_solve(inst, model=untrained, topk=4, **kw)
    c = F.fsp_solve(inst, **kw)
    for k in KEYS[:-1]:
        assert a[k] == b[k] == c[k], k
    assert a["early_pruned"] > b["early_pruned"], (a["early_pruned"], b["early_pruned"])
    assert c["early_pruned"] == 0
    # the family counts: the same searches close the same families by their
    # one-machine bounds; only the learned order closes any by predicted
    # pairs, and every family it closes that way skips its exact pairs
    assert a["families_closed_lb1"] == b["families_closed_lb1"] == c["families_closed_lb1"] > 0
    assert c["families_closed_predicted"] == 0
    assert a["families_closed_predicted"] > b["families_closed_predicted"] >= 0
    assert a["exact_pair_evals"] <= c["exact_pair_evals"]


def test_trained_network_time_against_the_plain_orders(F, monkeypatch):
    """What the trained network buys in time, on a fixed node budget: the
    oracle checks the search (the learned search equals oracle.solve on a
    budget it finishes quickly); on a larger budget the three arms explore
    the same nodes, and the learned order (inference included) takes less
    time than the plain order bounded child by child, the paper's one bound
    per subproblem.  Against the plain order on the certified family kernel
    it is slower (the family kernel leaves little pair work to save; the
    counters of test_trained_network_cuts_more_than_untrained show it), so
    that ratio is reported, not asserted."""
    import torch
    n, m = 20, 20
    P = m * (m - 1) // 2
    p = inputs.instance(n, m, 6)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst)
    log = torch.zeros((200000, inst.stride), dtype=torch.uint8, device="cuda")
    F.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=8192, node_budget=200000, log_nodes=log)
    x, y = F.fsp_node_features(inst, log)
    net = F.Mlp(2 * m + 1, 128, P, seed=2)
    for it in range(400):
        s = (it * 4096) % (len(y) - 4096)
        net.train_step(x[s:s + 4096], y[s:s + 4096], lr=2e-3)
    small = dict(ub0=ub0, ub0_perm=perm0, pool_size=4096, node_budget=60000)
    a = F.fsp_solve(inst, model=net, topk=4, **small)
    ref = oracle.solve(p, ub0=ub0, pool=4096, node_budget=60000, ub0_perm=[int(v) for v in perm0])
    assert a["cmax"] == ref["cmax"] and a["nodes_bounded"] == ref["bounded"]
    assert a["nodes_pruned"] == ref["pruned"] and a["iterations"] == ref["iterations"]
    big = dict(ub0=ub0, ub0_perm=perm0, pool_size=1 << 17, node_budget=20_000_000)
    for _ in range(2):  # warm-up
        F.fsp_solve(inst, model=net, topk=4, **big)
    learned = F.fsp_solve(inst, model=net, topk=4, **big)
    family = F.fsp_solve(inst, **big)
    monkeypatch.setenv("FSP_FAMILY", "0")
    F.fsp_solve(inst, **big)
    per_child = F.fsp_solve(inst, **big)
    for k in KEYS[:-1]:
        assert learned[k] == family[k] == per_child[k], k
    assert learned["time_ms"] < per_child["time_ms"], (learned["time_ms"], per_child["time_ms"])
    print(f"learned {learned['time_ms']:.1f} ms, plain family {family['time_ms']:.1f} ms, "
          f"plain per child {per_child['time_ms']:.1f} ms")
