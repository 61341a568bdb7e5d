"""Pins of the oracle's bidirectional branching (oracle/fsp_oracle.c,
orc_*2 / orc_solve_bidir), none of them re-using its code: delivery times
against a longest-path recurrence over the suffix written here, the bound
against every completion (brute force), its two reductions (empty suffix:
the forward bound; nothing left: the makespan), the solver's optimum against
brute force over all n! schedules, and its pool-1 counters against a
recursive textbook depth-first search.  No GPU."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1206_4973_gb300 import inputs


def simulate(p, seq):
    """Makespan of a permutation schedule: completion times row by row."""
    m = p.shape[1]
    c = [0] * m
    for j in seq:
        for k in range(m):
            c[k] = max(c[k], c[k - 1] if k else 0) + int(p[j][k])
    return c[-1]


def longest_path_from(p, suffix, k):
    """Longest monotone path (right along a job's machines, down to the next
    job) from (suffix[0], machine k) to (suffix[-1], machine m-1)."""
    m = p.shape[1]
    G = np.zeros((len(suffix), m), np.int64)
    for i, j in enumerate(suffix):
        for h in range(k, m):
            best = 0
            if i > 0:
                best = max(best, G[i - 1][h])
            if h > k:
                best = max(best, G[i][h - 1])
            G[i][h] = best + int(p[j][h])
    return int(G[-1][m - 1])


def rand_split(n, rng):
    perm = rng.permutation(n).astype(np.uint8)
    d1 = int(rng.integers(0, n + 1))
    d2 = int(rng.integers(0, n - d1 + 1))
    return perm, d1, d2


@pytest.mark.parametrize("n,m,seed", [(6, 4, 1), (9, 5, 2), (12, 3, 3), (7, 8, 4)])
def test_delivery_times_are_longest_paths(n, m, seed):
    p = inputs.instance(n, m, seed)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        perm, d1, d2 = rand_split(n, rng)
        if d2 == 0:
            continue
        _, _, _, D = oracle.lb2_parts(p, perm, d1, d2)
        suffix = list(perm[n - d2:])
        assert [int(x) for x in D] == [longest_path_from(p, suffix, k) for k in range(m)]


@pytest.mark.parametrize("n,m,seed", [(6, 4, 11), (8, 5, 12), (10, 3, 13)])
def test_bound_with_nothing_left_is_the_makespan(n, m, seed):
    p = inputs.instance(n, m, seed)
    rng = np.random.default_rng(seed)
    for _ in range(25):
        perm = rng.permutation(n).astype(np.uint8)
        d1 = int(rng.integers(0, n + 1))
        lb, _, _, _ = oracle.lb2_parts(p, perm, d1, n - d1)
        assert lb == simulate(p, perm)


@pytest.mark.parametrize("n,m,seed", [(7, 4, 21), (9, 6, 22), (5, 3, 23)])
def test_empty_suffix_gives_the_forward_bound(n, m, seed):
    p = inputs.instance(n, m, seed)
    rng = np.random.default_rng(seed)
    for _ in range(25):
        perm = rng.permutation(n).astype(np.uint8)
        d = int(rng.integers(0, n + 1))
        assert oracle.lb2_parts(p, perm, d, 0)[0] == oracle.lb(p, perm, d)


@pytest.mark.parametrize("n,m,seed", [(6, 3, 31), (7, 4, 32), (6, 6, 33), (8, 3, 34)])
def test_bound_is_valid_against_every_completion(n, m, seed):
    p = inputs.instance(n, m, seed)
    rng = np.random.default_rng(seed)
    for _ in range(15):
        perm, d1, d2 = rand_split(n, rng)
        lb, lb1, pairs, _ = oracle.lb2_parts(p, perm, d1, d2)
        mid = list(perm[d1:n - d2])
        best = min(simulate(p, list(perm[:d1]) + list(o) + list(perm[n - d2:]))
                   for o in itertools.permutations(mid)) if mid else simulate(p, perm)
        assert lb1 <= lb <= best
        assert max(pairs.max(initial=0), lb1) == lb


@pytest.mark.parametrize("n,m,seed", [(5, 3, 41), (7, 4, 42), (8, 5, 43), (9, 3, 44), (6, 7, 45)])
@pytest.mark.parametrize("pool", [1, 7, 64, 4096])
def test_bidirectional_solver_reaches_the_brute_force_optimum(n, m, seed, pool):
    p = inputs.instance(n, m, seed)
    r = oracle.solve_bidir(p, pool=pool)
    best, _ = oracle.bruteforce(p)
    assert r["status"] == oracle.OK and r["cmax"] == best
    assert simulate(p, r["perm"]) == best


def textbook_dfs(p):
    """Recursive depth-first search with the same rules at pool size 1:
    children by increasing job index, forward when d1 <= d2, one-job-left
    children are complete schedules, the UB moves after each parent's
    children are bounded, survivors are visited in order without a re-check."""
    n, m = p.shape
    st = dict(bounded=0, branched=0, pruned=0, leaves=0, iterations=0, incumbent_updates=0)
    ub = [oracle.INF]

    def visit(prefix, rest, suffix):
        st["branched"] += 1
        st["iterations"] += 1
        forward = len(prefix) <= len(suffix)
        kids = []
        for j in sorted(rest):
            left = [x for x in sorted(rest) if x != j]
            pre, suf = (prefix + [j], suffix) if forward else (prefix, [j] + suffix)
            perm = np.array(pre + left + suf, np.uint8)
            if len(left) == 1:
                kids.append((pre, left, suf, simulate(p, list(perm)), True))
            else:
                kids.append((pre, left, suf, oracle.lb2_parts(p, perm, len(pre), len(suf))[0], False))
        st["bounded"] += len(kids)
        before = ub[0]
        for pre, left, suf, v, leaf in kids:
            if leaf:
                st["leaves"] += 1
                ub[0] = min(ub[0], v)
        if ub[0] < before:
            st["incumbent_updates"] += 1
        live = []
        for pre, left, suf, v, leaf in kids:
            if leaf:
                continue
            if v < ub[0]:
                live.append((pre, left, suf))
            else:
                st["pruned"] += 1
        for pre, left, suf in live:
            visit(pre, left, suf)

    visit([], list(range(n)), [])
    return ub[0], st


@pytest.mark.parametrize("n,m,seed", [(6, 3, 51), (7, 4, 52), (8, 3, 53)])
def test_pool_one_counts_equal_a_textbook_dfs(n, m, seed):
    p = inputs.instance(n, m, seed)
    r = oracle.solve_bidir(p, pool=1)
    cmax, st = textbook_dfs(p)
    assert r["cmax"] == cmax
    for k, v in st.items():
        assert r[k] == v, k


@pytest.mark.parametrize("n,m,seed", [(6, 4, 61), (7, 3, 62), (6, 5, 63)])
def test_pair_values_from_their_definition(n, m, seed):
    """Every pair value: the lagged two-machine recurrence over U at its best
    order (brute force over the orders of U, which Johnson's rule attains),
    from the prefix's release times, plus the tail after machine l: the
    suffix's delivery time or the smallest remaining tail, whichever is
    larger."""
    p = inputs.instance(n, m, seed)
    rng = np.random.default_rng(seed)
    for _ in range(12):
        perm, d1, d2 = rand_split(n, rng)
        mid = list(perm[d1:n - d2])
        if not mid:
            continue
        _, _, pairs, _ = oracle.lb2_parts(p, perm, d1, d2)
        C = [0] * m
        for j in perm[:d1]:
            for k in range(m):
                C[k] = max(C[k], C[k - 1] if k else 0) + int(p[j][k])
        suffix = list(perm[n - d2:])
        idx = 0
        for k in range(m):
            for l in range(k + 1, m):
                best = None
                for o in itertools.permutations(mid):
                    tk, tl = C[k], C[l]
                    for j in o:
                        tk += int(p[j][k])
                        tl = max(tl, tk + int(p[j][k + 1:l].sum())) + int(p[j][l])
                    best = tl if best is None else min(best, tl)
                qmin = min(int(p[j][l + 1:].sum()) for j in mid)
                D = longest_path_from(p, suffix, l) if suffix else 0
                assert pairs[idx] == best + max(D, qmin), (k, l)
                idx += 1
