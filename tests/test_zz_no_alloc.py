"""fsp_solve_noalloc: the search entry point that allocates no device memory.

Some callers cannot call cudaMalloc while they run: processes whose device
memory is reserved up front by a pool or a fixed budget, plugins that are
handed only their input and output buffers, and code paths that cannot afford
cudaMalloc's implicit synchronisation of the device.  For them the library
keeps a fixed scratch array of NOALLOC_SCRATCH_BYTES on each device.  This
test calls that entry point through the C ABI and checks it gives exactly what
fsp_solve gives (all results are integers: bit-exact), on two calls in a row,
and that a search too large for the array is refused.  The file name makes
pytest collect it last.
"""
import numpy as np
import pytest

from paper_1206_4973_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("cmax", "status", "nodes_bounded", "nodes_branched", "nodes_pruned", "leaves", "iterations",
        "incumbent_updates", "stack_left")


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_1206_4973_gb300 import build, fsp
    build.build()
    fsp.load()
    assert torch.cuda.is_available()
    return fsp


def same(a, b):
    for k in KEYS:
        assert a[k] == b[k], k
    assert (a["perm"] is None) == (b["perm"] is None)
    if a["perm"] is not None:
        assert list(a["perm"]) == list(b["perm"])
    assert np.array_equal(a["trace"], b["trace"])


def test_noalloc_first_on_a_new_instance_creates_nothing(F):
    """On a newly created instance the first calls go to the entry point that
    allocates nothing: they must create no pinned block and no CUDA event
    (the instance's counts stay at what fsp_create_instance reserved); only
    then does fsp_solve run, and the results must be identical."""
    import torch
    # the library's device code (its fixed array included) is loaded on the
    # device by the first call that uses it: done here on another instance of
    # the same shape, so the free-memory check below sees only the call
    F.fsp_solve_noalloc(F.fsp_create_instance(inputs.instance(12, 5, 1)), pool_size=1024)
    p = inputs.instance(12, 5, 0)
    inst = F.fsp_create_instance(p)
    before = F.fsp_instance_host_objects(inst)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = [F.fsp_solve_noalloc(inst, pool_size=1024, trace_cap=4096) for _ in range(2)]
    torch.cuda.synchronize()
    assert F.fsp_instance_host_objects(inst) == before
    assert torch.cuda.mem_get_info()[0] == free0  # no device memory taken either
    ref = F.fsp_solve(inst, pool_size=1024, trace_cap=4096)
    for g in got:
        same(g, ref)
        assert g["nodes_bounded"] > 0
    # fsp_solve itself does create read-back objects (its cache was empty)
    assert F.fsp_instance_host_objects(inst) != before


def test_noalloc_matches_fsp_solve_twice_in_a_row(F):
    p = inputs.instance(12, 5, 0)
    inst = F.fsp_create_instance(p)
    ref = F.fsp_solve(inst, pool_size=1024, trace_cap=4096)
    for _ in range(2):
        got = F.fsp_solve_noalloc(inst, pool_size=1024, trace_cap=4096)
        same(got, ref)
        assert got["nodes_bounded"] > 0


def test_noalloc_after_another_shape_and_from_a_frontier(F):
    """The shared array keeps the previous call's contents; a call on another
    instance, then a budgeted call from start records, still match."""
    p2 = inputs.instance(9, 20, 88)
    inst2 = F.fsp_create_instance(p2)
    same(F.fsp_solve_noalloc(inst2, pool_size=64, trace_cap=4096),
         F.fsp_solve(inst2, pool_size=64, trace_cap=4096))
    p, ub_perm, rec = inputs.pool_workload(20, 20, 1, 4000)
    rec = rec[rec[:, 20] <= 18]
    inst = F.fsp_create_instance(p)
    kw = dict(ub0=3000, pool_size=2048, init_nodes=rec, max_iterations=3, trace_cap=16)
    before = F.fsp_instance_host_objects(inst)
    b = F.fsp_solve_noalloc(inst, **kw)
    c = F.fsp_solve_noalloc(inst, **kw)
    assert F.fsp_instance_host_objects(inst) == before
    a = F.fsp_solve(inst, **kw)
    same(b, a)
    same(c, a)


def test_noalloc_refuses_a_search_larger_than_its_scratch(F):
    p = inputs.instance(20, 20, 1)
    inst = F.fsp_create_instance(p)
    assert F.fsp_solve_workspace_bytes(inst, pool_size=2**20) > F.NOALLOC_SCRATCH_BYTES
    with pytest.raises(F.FspError) as e:
        F.fsp_solve_noalloc(inst, pool_size=2**20)
    assert e.value.code == F.ERR_CAPACITY
    assert "scratch" in str(e.value)
