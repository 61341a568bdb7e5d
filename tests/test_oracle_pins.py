"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check uses a different computation from the oracle's: the longest-path
characterisation of the makespan, brute force over orders or completions,
Johnson's theorem at m = 2, a recursive DFS, and the order-free set of nodes a
search with a fixed incumbent must bound.  A dropped term, a wrong sign or
index, or a swapped operand in the oracle fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1206_4973_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --
def longest_path_makespan(p, perm):
    """Makespan as the heaviest monotone lattice path through the grid of
    (position, machine) operation times (permutation flow shop, Sec. II-B)."""
    n_, m = len(perm), p.shape[1]
    best = 0
    # a path is fixed by the positions at which it steps to the next machine
    for cuts in itertools.combinations_with_replacement(range(n_), m - 1):
        s, pos = 0, 0
        bounds = list(cuts) + [n_ - 1]
        for k in range(m):
            end = bounds[k]
            for i in range(pos, end + 1):
                s += int(p[perm[i], k])
            pos = end
        best = max(best, s)
    return best


def release_time_brute(p, prefix, k):
    """Completion time on machine k of the prefix = longest path on machines 0..k."""
    if len(prefix) == 0:
        return 0
    return longest_path_makespan(p[:, : k + 1], list(prefix))


def two_machine_value(a, b, lag, order, ck, cl):
    """Schedule the jobs in `order` on machines k then l (k from ck, l from cl,
    job j may start on l only lag_j after it ends on k); return the end on l."""
    tk, tl = ck, cl
    for j in order:
        start_k = tk
        tk = start_k + a[j]
        start_l = max(tl, tk + lag[j])
        tl = start_l + b[j]
    return tl


def rand_nodes(n, count, seed):
    rng = inputs.SplitMix64(seed)
    out = []
    for _ in range(count):
        perm = inputs.permutation(n, rng)
        d = int(rng.take_hi(1)[0] % np.uint64(n + 1))
        out.append((perm, d))
    return out


# ------------------------------------------------------------- makespan ---
def test_makespan_hand_worked():
    # two jobs, two machines: job0 = (3, 2), job1 = (1, 4)
    # order (0, 1): M1 busy [0,3) then [3,4); M2 [3,5) then [5,9)  -> 9
    # order (1, 0): M1 [0,1) then [1,4);  M2 [1,5) then [5,7)      -> 7
    p = np.array([[3, 2], [1, 4]], np.int32)
    assert oracle.makespan(p, [0, 1]) == 9
    assert oracle.makespan(p, [1, 0]) == 7
    # one job: the sum of its times
    assert oracle.makespan(np.array([[5, 6, 7]], np.int32), [0]) == 18


@pytest.mark.parametrize("n,m,seed", [(3, 3, 11), (4, 5, 12), (6, 3, 13), (5, 4, 14)])
def test_makespan_equals_longest_path(n, m, seed):
    p = inputs.instance(n, m, seed)
    rng = inputs.SplitMix64(seed + 1000)
    for _ in range(6):
        perm = inputs.permutation(n, rng)
        assert oracle.makespan(p, perm) == longest_path_makespan(p, list(perm))


def test_release_times_match_truncated_longest_path():
    p = inputs.instance(6, 5, 21)
    for perm, d in rand_nodes(6, 8, 22):
        C = oracle.release_times(p, perm, d)
        for k in range(5):
            assert C[k] == release_time_brute(p, perm[:d], k)


# ------------------------------------------------ two-machine sub-bounds ---
@pytest.mark.parametrize("n,m,seed", [(7, 4, 31), (6, 5, 32), (7, 3, 33)])
def test_pair_bound_is_optimal_two_machine_value(n, m, seed):
    """LB_kl = min over every order of the remaining jobs of the lagged
    two-machine schedule on (k, l), plus the smallest tail after l."""
    p = inputs.instance(n, m, seed)
    for perm, d in rand_nodes(n, 10, seed + 1):
        prefix, U = list(perm[:d]), list(perm[d:])
        _, _, pv = oracle.lb_parts(p, perm, d)
        C = [release_time_brute(p, prefix, k) for k in range(m)]
        for idx, (k, l) in enumerate(oracle.pairs(m)):
            a, b = p[:, k], p[:, l]
            lag = p[:, k + 1:l].sum(axis=1)
            qmin_l = min((int(p[j, l + 1:].sum()) for j in U), default=0)
            best = min(two_machine_value(a, b, lag, o, C[k], C[l])
                       for o in itertools.permutations(U)) if U else C[l]
            assert pv[idx] == best + qmin_l, (perm, d, k, l)


@pytest.mark.parametrize("crafted", [False, True])
def test_one_machine_bound_definition(crafted):
    """LB1 = max_k release + remaining work + smallest tail, written from the
    definition with brute-force release times.  The crafted instance makes
    machine 0 the bottleneck, so the tail term decides LB1."""
    n, m = 6, 4
    p = inputs.instance(n, m, 41)
    if crafted:
        p = p % 5 + 1
        p[:, 0] += 90
    for perm, d in rand_nodes(n, 10, 42):
        U = list(perm[d:])
        lb, lb1, pv = oracle.lb_parts(p, perm, d)
        want = 0
        for k in range(m):
            ck = release_time_brute(p, list(perm[:d]), k)
            sk = sum(int(p[j, k]) for j in U)
            qk = min((int(p[j, k + 1:].sum()) for j in U), default=0)
            want = max(want, ck + sk + qk)
        assert lb1 == want
        assert lb == max(lb1, int(pv.max()))


def test_johnson_orders_are_permutations_with_rule():
    p = inputs.instance(9, 6, 43)
    q, lag, order = oracle.tables(p)
    for idx, (k, l) in enumerate(oracle.pairs(6)):
        o = list(order[idx])
        assert sorted(o) == list(range(9))
        a, b = p[:, k], p[:, l]
        first = [j for j in o if a[j] <= b[j]]
        # set A precedes set B
        assert o[: len(first)] == first


def test_johnson_tie_break_hand_worked():
    """Equal sort keys inside set A and inside set B go smaller job index
    first, and a job with a == b belongs to set A (worked by hand).
    Two machines: A = {a <= b} by increasing a: j1 (2), j0 (3), j2 (3),
    j6 (4); B = {a > b} by decreasing b: j4 (5), j3 (2), j5 (2)."""
    p = np.array([[3, 5], [2, 9], [3, 4], [7, 2], [6, 5], [8, 2], [4, 4]], np.int32)
    _, lag, order = oracle.tables(p)
    assert list(lag[0]) == [0] * 7
    assert list(order[0]) == [1, 0, 2, 6, 4, 3, 5]
    # Three machines, pair (0, 2) (index 1), lag = the time on machine 1:
    # A by increasing a + lag: j2 (1+2=3), j0 (2+3=5), j1 (4+1=5), j5 (5+4=9);
    # B by decreasing b + lag: j3 (1+2=3), j4 (2+1=3).
    p = np.array([[2, 3, 9], [4, 1, 6], [1, 2, 7], [9, 2, 1], [8, 1, 2], [5, 4, 5]], np.int32)
    _, lag, order = oracle.tables(p)
    assert list(lag[1]) == [3, 1, 2, 2, 1, 4]
    assert list(order[1]) == [2, 0, 1, 5, 3, 4]


# ------------------------------------------------------------ the bound ---
@pytest.mark.parametrize("n,m,seed", [(6, 3, 51), (7, 4, 52), (5, 6, 53), (7, 5, 54)])
def test_bound_is_valid_and_exact_at_the_leaves(n, m, seed):
    p = inputs.instance(n, m, seed)
    for perm, d in rand_nodes(n, 14, seed + 7):
        lb = oracle.lb(p, perm, d)
        best = min(oracle.makespan(p, list(perm[:d]) + list(o))
                   for o in itertools.permutations(perm[d:]))
        assert lb <= best
        if d >= n - 1:
            assert lb == best == longest_path_makespan(p, list(perm))


@pytest.mark.parametrize("seed", [61, 62, 63, 64])
def test_bound_exact_at_m2(seed):
    """With two machines the pair relaxation is the problem itself (Johnson's
    theorem): every node's bound equals its best completion."""
    n = 7
    p = inputs.instance(n, 2, seed)
    opt, _ = oracle.bruteforce(p)
    assert oracle.lb(p, np.arange(n), 0) == opt
    for perm, d in rand_nodes(n, 12, seed + 3):
        best = min(oracle.makespan(p, list(perm[:d]) + list(o))
                   for o in itertools.permutations(perm[d:]))
        assert oracle.lb(p, perm, d) == best


def test_bound_pool_matches_single_node_and_rejects_bad_records():
    n, m = 8, 5
    p, _, nodes = inputs.pool_workload(n, m, 71, 64)
    lbs = oracle.bound_pool(p, nodes)
    for t in range(64):
        assert lbs[t] == oracle.lb(p, nodes[t, :n], nodes[t, n])
    bad = nodes.copy()
    bad[3, 0] = bad[3, 1]  # repeated job
    with pytest.raises(ValueError):
        oracle.bound_pool(p, bad)
    bad = nodes.copy()
    bad[5, n] = n + 1  # depth > n
    with pytest.raises(ValueError):
        oracle.bound_pool(p, bad)


# ----------------------------------------- bound variant: smallest heads ---
def test_head_variant_hand_worked():
    """Job 0 scheduled (times 5, 1, 1); jobs 1 (3, 4, 9) and 2 (4, 3, 8) remain.
    Prefix release times C = (5, 6, 7).  A remaining job reaches machine 1 no
    earlier than 5 + min(3, 4) = 8 and machine 2 no earlier than 8 + min(4, 3)
    = 11, so the machine-2 one-machine term rises from 7 + 17 = 24 to 11 + 17
    = 28 (tails: job 1 (13, 9, 0), job 2 (11, 8, 0)); the best completion is
    29 either way round."""
    p = np.array([[5, 1, 1], [3, 4, 9], [4, 3, 8]], np.int32)
    perm = np.array([0, 1, 2], np.uint8)
    _, lb1_base, _ = oracle.lb_parts(p, perm, 1)
    lb_head, lb1_head, _ = oracle.lb_parts(p, perm, 1, bound=1)
    assert lb1_base == 24 and lb1_head == 28
    assert lb_head <= 29 == min(longest_path_makespan(p, [0, 1, 2]), longest_path_makespan(p, [0, 2, 1]))


@pytest.mark.parametrize("n,m,seed", [(6, 3, 141), (7, 4, 142), (5, 6, 143), (7, 5, 144)])
def test_head_variant_is_valid_dominant_and_exact_at_the_leaves(n, m, seed):
    p = inputs.instance(n, m, seed)
    for perm, d in rand_nodes(n, 14, seed + 7):
        base = oracle.lb(p, perm, d)
        head = oracle.lb(p, perm, d, bound=1)
        best = min(oracle.makespan(p, list(perm[:d]) + list(o))
                   for o in itertools.permutations(perm[d:]))
        assert base <= head <= best
        if d >= n - 1:
            assert head == best == longest_path_makespan(p, list(perm))
    # the one-machine part is where the heads act (the pair bounds already
    # carry most of them): it rises on some nodes and never falls
    rises = 0
    for perm, d in rand_nodes(n, 200, seed + 8):
        lb1_base = oracle.lb_parts(p, perm, d)[1]
        lb1_head = oracle.lb_parts(p, perm, d, bound=1)[1]
        assert lb1_head >= lb1_base
        rises += lb1_head > lb1_base
    assert rises > 0


@pytest.mark.parametrize("seed", [151, 152])
def test_head_variant_exact_at_m2(seed):
    """At m = 2 the base bound is already the best completion (Johnson), so the
    stronger variant must equal it."""
    n = 7
    p = inputs.instance(n, 2, seed)
    for perm, d in rand_nodes(n, 12, seed + 3):
        assert oracle.lb(p, perm, d, bound=1) == oracle.lb(p, perm, d)


@pytest.mark.parametrize("n,m,seed", [(6, 3, 161), (7, 5, 162), (8, 4, 163), (9, 3, 164)])
@pytest.mark.parametrize("pool", [1, 7, 1024])
def test_head_variant_solver_reaches_brute_force_optimum(n, m, seed, pool):
    p = inputs.instance(n, m, seed)
    opt, _ = oracle.bruteforce(p)
    head = oracle.solve(p, pool=pool, bound=1)
    base = oracle.solve(p, pool=pool)
    assert head["status"] == oracle.OK and head["cmax"] == opt
    assert oracle.makespan(p, head["perm"]) == opt
    if pool == 1:  # depth-first one node at a time: a stronger bound never bounds more nodes
        assert head["bounded"] <= base["bounded"]

# ----------------------------------------------------------- the search ---
@pytest.mark.parametrize("n,m,seed", [(2, 3, 80), (5, 2, 81), (6, 3, 82), (7, 5, 83), (8, 4, 84),
                                      (8, 2, 85), (9, 3, 86)])
@pytest.mark.parametrize("pool", [1, 3, 7, 1024])
def test_solver_reaches_brute_force_optimum(n, m, seed, pool):
    p = inputs.instance(n, m, seed)
    opt, _ = oracle.bruteforce(p)
    res = oracle.solve(p, pool=pool, trace_cap=100000)
    assert res["status"] == oracle.OK
    assert res["cmax"] == opt
    assert sorted(res["perm"]) == list(range(n))
    assert oracle.makespan(p, res["perm"]) == opt
    tr = res["trace"]
    # a pool never holds more children than its size unless one parent alone overflows it
    assert np.all((tr[:, 1] <= pool) | (tr[:, 0] == 1))
    assert tr[:, 1].sum() == res["bounded"] and tr[:, 0].sum() == res["branched"]
    assert res["bounded"] == res["leaves"] + res["pruned"] + tr[:, 2].sum()


def textbook_dfs(p, n, ub0):
    """Recursive depth-first B&B: branch a node, bound all its children, let
    complete children improve the incumbent in order, drop children with
    bound >= incumbent, recurse into the rest in order."""
    st = {"ub": ub0, "bounded": 0, "branched": 0, "perm": None}

    def visit(prefix, rem):
        st["branched"] += 1
        kids = []
        for j in sorted(rem):
            child = prefix + [j]
            rest = sorted(set(rem) - {j})
            kids.append((child, rest, oracle.lb(p, child + rest, len(child))))
        st["bounded"] += len(kids)
        for child, rest, v in kids:
            if len(rest) == 1 and v < st["ub"]:
                st["ub"], st["perm"] = v, child + rest
        keep = [(c, r, v) for c, r, v in kids if len(r) > 1 and v < st["ub"]]
        for c, r, _ in keep:
            visit(c, r)

    visit([], list(range(n)))
    return st


@pytest.mark.parametrize("n,m,seed", [(6, 3, 91), (7, 4, 92), (8, 3, 93)])
def test_pool_one_equals_recursive_dfs(n, m, seed):
    p = inputs.instance(n, m, seed)
    ref = textbook_dfs(p, n, oracle.INF)
    res = oracle.solve(p, pool=1)
    assert (res["bounded"], res["branched"], res["cmax"]) == (ref["bounded"], ref["branched"], ref["ub"])
    assert list(res["perm"]) == ref["perm"]


@pytest.mark.parametrize("n,m,seed", [(7, 4, 101), (8, 3, 102), (8, 5, 103)])
def test_fixed_incumbent_explores_order_free_set(n, m, seed):
    """With ub0 = optimum the incumbent never changes, so the nodes bounded are
    exactly the children of every node whose ancestors all bound below it,
    whatever the pool size."""
    p = inputs.instance(n, m, seed)
    opt, _ = oracle.bruteforce(p)
    bounded = branched = 0
    frontier = [([], list(range(n)))]
    while frontier:
        prefix, rem = frontier.pop()
        branched += 1
        for j in rem:
            child, rest = prefix + [j], [x for x in rem if x != j]
            bounded += 1
            if len(rest) > 1 and oracle.lb(p, child + rest, len(child)) < opt:
                frontier.append((child, rest))
    for pool in (1, 2, 5, 16, 4096):
        res = oracle.solve(p, ub0=opt, pool=pool)
        assert (res["bounded"], res["branched"]) == (bounded, branched)
        assert res["cmax"] == opt and res["incumbent_updates"] == 0 and res["perm"] is None


def test_solver_edge_cases():
    p1 = np.array([[4, 5, 6]], np.int32)
    r = oracle.solve(p1)
    assert r["cmax"] == 15 and list(r["perm"]) == [0] and r["iterations"] == 0
    p = inputs.instance(6, 3, 111)
    opt, _ = oracle.bruteforce(p)
    r = oracle.solve(p, ub0=opt - 1)  # nothing beats a UB below the optimum
    assert r["cmax"] == opt - 1 and r["perm"] is None
    r = oracle.solve(p, pool=4, node_budget=10)
    assert r["status"] == oracle.INCOMPLETE and r["bounded"] >= 10


def test_schedule_replay_equals_fixed_pool():
    p = inputs.instance(8, 4, 121)
    a = oracle.solve(p, pool=9)
    b = oracle.solve(p, pool=1, schedule=[9])
    assert {k: a[k] for k in oracle.STATS} == {k: b[k] for k in oracle.STATS}


# ---------------------------------------------------------------- NEH -----
@pytest.mark.parametrize("n,m,seed", [(1, 3, 130), (2, 2, 131), (7, 4, 132), (8, 5, 133)])
def test_neh_is_a_valid_upper_bound(n, m, seed):
    p = inputs.instance(n, m, seed)
    c, perm = oracle.neh(p)
    assert sorted(perm) == list(range(n))
    assert c == oracle.makespan(p, perm) == longest_path_makespan(p, list(perm))
    assert c >= oracle.bruteforce(p)[0]


def test_neh_hand_worked():
    # totals: job0 = 5, job1 = 5, job2 = 9 -> insertion order 2, 0, 1
    # [2] -> insert 0: [0,2] = 12, [2,0] = 11 -> [2,0]
    # insert 1 into [2,0]: [1,2,0] = 12, [2,1,0] = 15, [2,0,1] = 15 -> [1,2,0]
    p = np.array([[3, 2], [1, 4], [4, 5]], np.int32)
    c, perm = oracle.neh(p)
    assert list(perm) == [1, 2, 0] and c == 12


def test_neh_hand_worked_order_and_ties():
    """Decreasing total time fixes the insertion order, and equal partial
    makespans go to the earliest position (worked by hand, two machines:
    C1 = running sum of a, C2 = max(C2, C1) + b)."""
    # totals: job0 = 6, job1 = 9, job2 = 2 -> insertion order 1, 0, 2
    # [1] -> insert 0: [0,1] = 12, [1,0] = 12 -> tie, earliest: [0,1]
    # insert 2: [2,0,1] = 13, [0,2,1] = 13, [0,1,2] = 13 -> earliest: [2,0,1]
    # (increasing totals would give [1,0,2]; latest ties would give [1,0,2])
    p = np.array([[3, 3], [4, 5], [1, 1]], np.int32)
    c, perm = oracle.neh(p)
    assert list(perm) == [2, 0, 1] and c == 13
    # two identical jobs: order 0, 1 (equal totals, smaller index first); both
    # positions give 3, so job 1 goes in front
    c, perm = oracle.neh(np.array([[1, 1], [1, 1]], np.int32))
    assert list(perm) == [1, 0] and c == 3


# --------------------------------------------------------- golden files ---
def test_golden_files_reproduce():
    """tests/golden/*.json were written by tests/golden/make_golden.py from the
    oracle alone; the oracle must still reproduce them."""
    for name in sorted(os.listdir(GOLDEN)):
        if not name.endswith(".json"):
            continue
        with open(os.path.join(GOLDEN, name)) as f:
            g = json.load(f)
        if g["kind"] == "solve":
            p = inputs.instance(g["n"], g["m"], g["seed"])
            r = oracle.solve(p, ub0=g["ub0"], pool=g["pool"])
            for k in oracle.STATS + ("cmax",):
                assert r[k] == g[k], (name, k)
            assert list(r["perm"]) == g["perm"]
        elif g["kind"] == "bound_pool":
            p, _, nodes = inputs.pool_workload(g["n"], g["m"], g["seed"], g["count"])
            lbs = oracle.bound_pool(p, nodes)
            assert lbs.tolist() == g["lb"]


# ---------------------------------------------------- checkpoint/resume ---
@pytest.mark.parametrize("pool,cut", [(1, 5), (16, 3), (256, 2)])
def test_resume_from_exported_stack_completes_the_search(pool, cut):
    """Stopping after `cut` iterations and resuming from the stack left, with
    the incumbent as ub0, reaches the same optimum with the same total work."""
    p = inputs.instance(9, 4, 151)
    full = oracle.solve(p, pool=pool)
    a = oracle.solve(p, pool=pool, max_iterations=cut, export_stack=True)
    assert a["status"] == oracle.INCOMPLETE and a["iterations"] == cut
    assert len(a["stack"]) == a["stack_left"] > 0
    b = oracle.solve(p, ub0=a["cmax"], pool=pool, init_nodes=a["stack"], ub0_perm=a["perm"])
    assert b["cmax"] == full["cmax"] == oracle.bruteforce(p)[0]
    for k in ("bounded", "branched", "pruned", "leaves", "iterations"):
        assert a[k] + b[k] == full[k], k
    assert list(b["perm"]) == list(full["perm"])


def test_init_nodes_are_validated():
    p = inputs.instance(6, 3, 161)
    rec = np.zeros((1, 16), np.uint8)
    rec[0, :6] = [0, 1, 2, 3, 4, 5]
    rec[0, 6] = 5  # depth n-1: a complete schedule, not a pending node
    with pytest.raises(ValueError):
        oracle.solve(p, init_nodes=rec)
    rec[0, 6] = 2
    rec[0, 1] = 0  # repeated job
    with pytest.raises(ValueError):
        oracle.solve(p, init_nodes=rec)


# ------------------------------------------------ learned-order network ---
def test_mlp_oracle_gradients_match_finite_differences():
    """With the bf16 rounding switched off the oracle's analytic gradients
    equal central differences of its loss (fp64): pins every backward term."""
    from oracle import mlp as om
    rng = np.random.default_rng(5)
    F, H, P, B = 7, 6, 5, 9
    params = {"W1": rng.normal(size=(F, H)), "b1": rng.normal(size=H) * 0.1, "W2": rng.normal(size=(H, H)),
              "b2": rng.normal(size=H) * 0.1, "W3": rng.normal(size=(H, P)), "b3": rng.normal(size=P) * 0.1}
    X = rng.normal(size=(B, F))
    y = rng.integers(0, P, size=B)
    _, g = om.loss_and_grads(params, X, y, rnd=om._same)
    eps = 1e-6
    for name, w in params.items():
        num = np.zeros_like(w)
        for idx in np.ndindex(*w.shape):
            old = w[idx]
            w[idx] = old + eps
            lp = om.loss(params, X, y, rnd=om._same)
            w[idx] = old - eps
            lm = om.loss(params, X, y, rnd=om._same)
            w[idx] = old
            num[idx] = (lp - lm) / (2 * eps)
        assert np.allclose(g[name], num, rtol=1e-5, atol=1e-7), name


def test_mlp_oracle_bf16_rounding_is_nearest_even():
    from oracle import mlp as om
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even significand (1)
    vals = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-8, -(2 + 2**-7), 1e-3, 65504.0])
    out = om.bf16(vals)
    assert out[0] == 1.0 and out[1] == 1.0 and out[2] == 1 + 2**-6 and out[3] == -2.0
    assert abs(out[4] - 1e-3) <= 1e-3 * 2**-8 and out[5] == 65536.0


@pytest.mark.parametrize("n,m,seed", [(7, 4, 171), (9, 6, 172)])
def test_feature_label_is_the_pair_that_gives_the_bound(n, m, seed):
    """The pair bounds dominate the one-machine bounds, so the labelled pair's
    bound is the node's bound; features are C/T, S/T, d/n."""
    from oracle import mlp as om
    p = inputs.instance(n, m, seed)
    T = np.float32(p.sum()) / np.float32(m)
    for perm, d in rand_nodes(n, 12, seed + 9):
        x, y = om.features(p, perm, d)
        lb, lb1, pv = oracle.lb_parts(p, perm, d)
        assert pv[y] == lb >= lb1 and y == int(np.flatnonzero(pv == pv.max())[0])
        assert x.dtype == np.float32 and x.shape == (2 * m + 1,)
        assert np.array_equal(x[:m], (oracle.release_times(p, perm, d).astype(np.float32) / T))
        rest = sorted(set(range(n)) - set(int(j) for j in perm[:d]))  # the remaining jobs, by definition
        S = np.array([sum(int(p[j, k]) for j in rest) for k in range(m)], np.float32)
        assert np.array_equal(x[m:2 * m], S / T)
        assert x[2 * m] == np.float32(d) / np.float32(n)


def test_mlp_oracle_forward_and_loss_hand_worked():
    """A 2 -> 2 -> 2 -> 2 network with small integer weights (every value exact
    in bf16), worked by hand: Z1 = x W1 + b1 = (1, -1), H1 = (1, 0);
    Z2 = H1 W2 + b2 = (2, 2) = H2; scores = H2 W3 + b3 = (3, 2).  Cross-entropy:
    label 0 gives log(1 + e^-1), label 1 gives log(1 + e)."""
    from oracle import mlp as om
    params = {"W1": np.array([[1.0, 0.0], [0.0, 1.0]]), "b1": np.array([0.0, -3.0]),
              "W2": np.array([[2.0, 1.0], [5.0, 5.0]]), "b2": np.array([0.0, 1.0]),
              "W3": np.array([[1.0, 0.0], [0.0, 1.0]]), "b3": np.array([1.0, 0.0])}
    X = np.array([[1.0, 2.0]])
    a = om.forward(params, X)
    assert np.array_equal(a["H1"], [[1.0, 0.0]]) and np.array_equal(a["H2"], [[2.0, 2.0]])
    assert np.array_equal(a["L"], [[3.0, 2.0]])
    assert abs(om.loss(params, X, np.array([0])) - np.log1p(np.exp(-1.0))) < 1e-12
    assert abs(om.loss(params, X, np.array([1])) - np.log1p(np.e)) < 1e-12
    X2 = np.vstack([X, X])
    want = (np.log1p(np.exp(-1.0)) + np.log1p(np.e)) / 2
    assert abs(om.loss(params, X2, np.array([0, 1])) - want) < 1e-12


def test_threaded_pool_bound_equals_the_serial_one():
    """The all-core baseline splits the nodes over host threads; every bound
    is the serial oracle's."""
    p, _, rec = inputs.pool_workload(20, 20, 1, 3001)
    want = oracle.bound_pool(p, rec)
    for threads in (1, 3, 0):
        got, used = oracle.bound_pool_threads(p, rec, threads)
        assert np.array_equal(got, want)
        assert used >= 1 and (threads == 0 or used == threads)
    bad = rec.copy()
    bad[5, 0] = bad[5, 1]
    with pytest.raises(ValueError):
        oracle.bound_pool_threads(p, bad, 2)
