"""NEH on the device and searches with the tuned pool size, against the
oracle: NEH bit-exact; a tuned search replayed on the oracle with the pool
sizes it chose gives the same counters, trace, optimum and permutation."""
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


@pytest.mark.parametrize("n,m,seed", [(1, 3, 9), (2, 2, 8), (7, 3, 1), (12, 5, 0), (20, 5, 2), (50, 5, 3),
                                      (100, 5, 4), (20, 10, 5), (50, 20, 7), (255, 3, 11)])
def test_neh_matches_oracle(F, n, m, seed):
    p = inputs.instance(n, m, seed)
    c, perm = F.fsp_neh(F.fsp_create_instance(p))
    c0, perm0 = oracle.neh(p)
    assert c == c0 and list(perm) == list(perm0)


@pytest.mark.parametrize("n,m,seed,window", [(12, 5, 0, 2), (20, 5, 2, 3), (10, 10, 87, 1)])
def test_tuned_search_replays_on_the_oracle(F, n, m, seed, window):
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    ub0, perm0 = F.fsp_neh(inst)
    got = F.fsp_solve(inst, ub0=ub0, ub0_perm=perm0, pool_size=0, tune_window=window,
                      schedule_cap=100000, trace_cap=100000)
    assert got["status"] == F.OK
    sched = got["schedule"]
    assert len(sched) == got["iterations"]
    assert sched[0] == 256 * 152 or sched[0] > 0  # starts at nodes-per-CTA x SMs
    ref = oracle.solve(p, ub0=ub0, ub0_perm=perm0, pool=1, schedule=sched, trace_cap=100000)
    for k in ("bounded", "branched", "pruned", "leaves", "iterations", "incumbent_updates"):
        assert got["nodes_" + k if k in ("bounded", "branched", "pruned") else k] == ref[k], k
    assert got["cmax"] == ref["cmax"]
    assert list(got["perm"]) == list(ref["perm"])
    assert np.array_equal(got["trace"], ref["trace"])
    assert got["tuned_pool"] in set(sched.tolist())
