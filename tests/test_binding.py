"""The Python binding's marshalling on CPU, against a stand-in for the two
solve entry points of the C ABI (no GPU): the options struct carries the
caller's arguments, the result dict carries every field the library wrote."""
import ctypes

import numpy as np
import pytest

from paper_1206_4973_gb300 import fsp


class _Inst:
    handle = ctypes.c_void_p(0)
    n, m, stride = 6, 3, 16


@pytest.fixture()
def fake(monkeypatch):
    real = fsp.load()
    seen = {}

    class Lib:
        def __getattr__(self, k):
            return getattr(real, k)

        def fsp_solve_workspace_bytes(self, inst, o):
            return 4096

        def fsp_solve(self, inst, ub0, cmax, perm, st, o):
            opt = ctypes.cast(o, ctypes.POINTER(fsp.fsp_options)).contents
            seen.update(ub0=ub0, pool=opt.pool_size, budget=opt.node_budget, init=opt.init_nodes,
                        init_count=opt.init_count, max_it=opt.max_iterations, profile=opt.profile,
                        workspace=opt.workspace, stream=opt.stream)
            ctypes.cast(cmax, ctypes.POINTER(ctypes.c_int32))[0] = 77
            p = ctypes.cast(perm, ctypes.POINTER(ctypes.c_int32))
            for i in range(6):
                p[i] = 5 - i
            s = ctypes.cast(st, ctypes.POINTER(fsp.fsp_stats)).contents
            s.nodes_bounded, s.iterations, s.incumbent_updates, s.bound_ms, s.tuned_warps = 123, 4, 1, 0.5, 8
            opt.out_count[0] = 9
            opt.log_count[0] = 0
            return fsp.INCOMPLETE

    monkeypatch.setattr(fsp, "_lib", Lib())
    return seen


def test_options_carry_the_arguments_and_results_come_back(fake):
    torch = pytest.importorskip("torch")
    ws = torch.empty(4096, dtype=torch.uint8)
    rec = np.zeros((3, 16), np.uint8)
    r = fsp.fsp_solve(_Inst(), ub0=900, pool_size=2048, node_budget=10**6, init_nodes=rec, max_iterations=5,
                      workspace=ws, profile=True, stream=0)
    assert fake["ub0"] == 900 and fake["pool"] == 2048 and fake["budget"] == 10**6
    assert fake["init"] == rec.ctypes.data and fake["init_count"] == 3 and fake["max_it"] == 5
    assert fake["profile"] == 1 and fake["workspace"] == ws.data_ptr() and not fake["stream"]
    assert r["status"] == fsp.INCOMPLETE and r["cmax"] == 77 and list(r["perm"]) == [5, 4, 3, 2, 1, 0]
    assert r["nodes_bounded"] == 123 and r["iterations"] == 4 and r["incumbent_updates"] == 1
    assert r["bound_ms"] == 0.5 and r["tuned_warps"] == 8 and r["stack_left"] == 9 and r["logged"] == 0
    for k in fsp.STATS + ("time_ms", "select_ms", "compact_ms", "infer_ms", "tuned_pool", "early_pruned"):
        assert k in r


def test_small_workspace_is_rejected_before_the_call(fake):
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        fsp.fsp_solve(_Inst(), workspace=torch.empty(100, dtype=torch.uint8), stream=0)
    assert "pool" not in fake
