"""GPU parity of the instance tables (K0) and the bounding kernel (K1) with the
CPU oracle: bit-exact int32 bounds, every kernel shape, ragged pools spanning
several CTAs, the edge depths 0, n-1 and n, malformed records, and the
full-size 20 x 20 bounding workload (sampled)."""
import numpy as np
import pytest

import oracle
from paper_1206_4973_gb300 import inputs

pytestmark = pytest.mark.gpu

# (n, m, seed): shapes cover mask words 1/2/4/8, machine templates 5/10/20,
# the any-m path, and Johnson entries in global memory (m = 64).
SHAPES = [(20, 20, 1), (12, 5, 0), (15, 10, 3), (7, 3, 4), (33, 5, 5), (50, 10, 6), (50, 20, 7),
          (100, 5, 8), (130, 5, 9), (20, 7, 10), (255, 3, 11), (2, 2, 12), (24, 64, 13), (100, 20, 14)]


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_1206_4973_gb300 import build, fsp
    build.build()
    fsp.load()
    assert torch.cuda.is_available()
    return fsp


def edge_pool(n, count, seed):
    rng = inputs.SplitMix64(seed)
    rec = inputs.random_prefix_pool(n, count, rng) if n >= 2 else np.zeros((count, 16), np.uint8)
    rec[::7, n] = 0
    rec[3::11, n] = n
    rec[5::13, n] = max(n - 1, 0)
    return rec


@pytest.mark.parametrize("n,m,seed", SHAPES)
def test_tables_match_oracle(F, n, m, seed):
    p = inputs.instance(n, m, seed)
    inst = F.fsp_create_instance(p)
    q, lag, order = F.fsp_instance_tables(inst)
    q0, lag0, order0 = oracle.tables(p)
    assert np.array_equal(q, q0)
    assert np.array_equal(lag, lag0)
    assert np.array_equal(order, order0)


@pytest.mark.parametrize("n,m,seed", SHAPES)
def test_bound_pool_matches_oracle(F, n, m, seed):
    import torch
    p = inputs.instance(n, m, seed)
    count = 3001 if n * m <= 2000 else 777
    rec = edge_pool(n, count, seed + 500)
    want = oracle.bound_pool(p, rec)
    inst = F.fsp_create_instance(p)
    nodes = torch.from_numpy(rec).cuda()
    got = F.fsp_bound_pool(inst, nodes).cpu().numpy()
    F.fsp_check_status(inst)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


def test_bound_pool_small_counts_and_offsets(F):
    import torch
    n, m = 20, 20
    p, _, rec = inputs.pool_workload(n, m, 1, 300)
    want = oracle.bound_pool(p, rec)
    inst = F.fsp_create_instance(p)
    nodes = torch.from_numpy(rec).cuda()
    for count in (0, 1, 31, 255, 256, 257):
        out = torch.full((300,), -7, dtype=torch.int32, device="cuda")
        F.fsp_bound_pool(inst, nodes, lb_out=out, count=count)
        got = out.cpu().numpy()
        assert np.array_equal(got[:count], want[:count])
        assert np.all(got[count:] == -7)  # nothing written past count
    # a pool that starts in the middle of a buffer (16-byte aligned records)
    sub = nodes[77:]
    got = F.fsp_bound_pool(inst, sub).cpu().numpy()
    assert np.array_equal(got, want[77:])


def test_malformed_records_are_flagged(F):
    import torch
    n, m = 12, 5
    p, _, rec = inputs.pool_workload(n, m, 3, 64)
    rec = rec.copy()
    rec[3, 0] = rec[3, 1]      # repeated job
    rec[9, n] = n + 1          # depth > n
    rec[20, 2] = n             # job id out of range
    inst = F.fsp_create_instance(p)
    got = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    assert got[3] == F.LB_INVALID and got[9] == F.LB_INVALID and got[20] == F.LB_INVALID
    good = np.ones(64, bool)
    good[[3, 9, 20]] = False
    assert np.array_equal(got[good], oracle.bound_pool(p, rec[good]))
    with pytest.raises(F.FspError) as e:
        F.fsp_check_status(inst)
    assert e.value.code == F.ERR_ARG
    F.fsp_check_status(inst)  # the flag was cleared


def test_bound_pool_argument_errors(F):
    import torch
    inst = F.fsp_create_instance(inputs.instance(8, 3, 1))
    with pytest.raises(F.FspError):  # negative count
        F._check(F.load().fsp_bound_pool(inst.handle, None, -1, 0, None, None))
    buf = torch.zeros((4, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FspError):  # misaligned records
        F._check(F.load().fsp_bound_pool(inst.handle, buf.data_ptr() + 1, 2, 0,
                                         torch.zeros(4, dtype=torch.int32, device="cuda").data_ptr(), 0))


@pytest.mark.parametrize("count", [2**12, 2**20])
def test_full_size_20x20_workload_sampled(F, count):
    """The 20 x 20 bounding workload as the benchmark runs it (seed 1): the
    whole pool bounded in one launch, a spread sample checked node by node."""
    import torch
    n, m = 20, 20
    p, ub_perm, rec = inputs.pool_workload(n, m, 1, count)
    inst = F.fsp_create_instance(p)
    got = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    F.fsp_check_status(inst)
    idx = np.unique(np.concatenate([np.arange(min(count, 512)), np.arange(count - 512, count),
                                    np.linspace(0, count - 1, 4096).astype(np.int64)]))
    want = oracle.bound_pool(p, rec[idx])
    assert np.array_equal(got[idx], want)
    # properties at any size: bounds are positive and never below the prefix makespan
    assert got.min() >= 1


@pytest.mark.parametrize("n,m,seed", [(20, 20, 1), (12, 5, 0), (33, 10, 21), (50, 20, 7), (15, 10, 22),
                                      (47, 5, 23), (63, 20, 24), (31, 20, 25), (9, 5, 26), (16, 10, 27),
                                      (31, 5, 28), (2, 5, 29)])
def test_every_kernel_family_agrees_with_oracle(F, n, m, seed, monkeypatch):
    """The shapes with a fast-path kernel, bounded by every kernel family:
    the default (two nodes per register where eligible), the per-node
    register kernel (FSP_BOUND_V2) and the generic one (FSP_BOUND_V1)."""
    import torch
    p = inputs.instance(n, m, seed)
    rec = edge_pool(n, 1500, seed + 77)
    want = oracle.bound_pool(p, rec)
    inst = F.fsp_create_instance(p)
    nodes = torch.from_numpy(rec).cuda()
    got = {"default": F.fsp_bound_pool(inst, nodes).cpu().numpy()}
    monkeypatch.setenv("FSP_BOUND_V2", "1")
    got["v2"] = F.fsp_bound_pool(inst, nodes).cpu().numpy()
    monkeypatch.delenv("FSP_BOUND_V2")
    monkeypatch.setenv("FSP_BOUND_V1", "1")
    got["v1"] = F.fsp_bound_pool(inst, nodes).cpu().numpy()
    for name, v in got.items():
        assert np.array_equal(v, want), (name, np.nonzero(v != want)[0][:10])


@pytest.mark.parametrize("warps", [1, 4, 8, 16])
def test_packed_kernel_cta_shapes(F, warps, monkeypatch):
    """The packed kernel gives the same bounds for every CTA shape, on a
    ragged pool (not a multiple of 32 nodes) spanning many warps."""
    import torch
    n, m = 20, 20
    p, _, rec = inputs.pool_workload(n, m, 1, 5003)
    want = oracle.bound_pool(p, rec)
    inst = F.fsp_create_instance(p)
    monkeypatch.setenv("FSP_POOL16_WARPS", str(warps))
    got = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,m,slices", [(20, 20, 1), (20, 20, 2), (20, 20, 3), (20, 20, 6), (15, 10, 2),
                                          (31, 10, 2), (12, 5, 1)])
def test_packed_kernel_pair_slices(F, n, m, slices, monkeypatch):
    """Teams of warps that split a group's passes over the machine pairs (the
    small-pool shape) give the same bounds as one warp per group, forward and
    bidirectional, on ragged pools of every size class: fewer nodes than one
    group, a few groups, and more groups than the teams resident at once."""
    import torch
    p = inputs.instance(n, m, 7)
    inst = F.fsp_create_instance(p)
    monkeypatch.setenv("FSP_POOL16_SLICES", str(slices))
    for count in (17, 300, 20011):
        _, _, rec = inputs.pool_workload(n, m, 7, count)
        want = oracle.bound_pool(p, rec)
        got = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
        assert np.array_equal(got, want), (count, np.nonzero(got != want)[0][:10])
    # bidirectional records: a suffix on every other node
    rng = np.random.default_rng(5)
    st2 = F.fsp_node_stride_bidir(n)
    rec2 = np.zeros((3001, st2), np.uint8)
    for t in range(rec2.shape[0]):
        rec2[t, :n] = rng.permutation(n)
        d1 = int(rng.integers(0, n - 1))
        d2 = int(rng.integers(0, n - d1)) if t % 2 else 0
        rec2[t, n], rec2[t, n + 1] = d1, d2
    want2 = oracle.bound_pool2(p, rec2)
    got2 = F.fsp_bound_pool_bidir(inst, torch.from_numpy(rec2).cuda()).cpu().numpy()
    assert np.array_equal(got2, want2), np.nonzero(got2 != want2)[0][:10]


def test_packed_kernel_extreme_times(F):
    """Instances at the edge of the packed kernel's 16-bit range
    ((n + m) * max p <= 16383) and just past it (the 32-bit kernels take
    over): processing times drawn near the largest allowed value."""
    import torch
    for n, m, pmax in ((20, 20, 409), (20, 20, 410), (31, 5, 455), (31, 5, 456), (12, 10, 744)):
        rng = np.random.default_rng(n * 1000 + pmax)
        p = rng.integers(max(1, pmax - 40), pmax + 1, size=(n, m)).astype(np.int32)
        p[0, 0] = pmax
        rec = edge_pool(n, 700, pmax)
        want = oracle.bound_pool(p, rec)
        inst = F.fsp_create_instance(p)
        got = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
        F.fsp_check_status(inst)
        assert np.array_equal(got, want), (n, m, pmax, np.nonzero(got != want)[0][:10])


def test_full_2e18_pool_elementwise(F):
    """The whole 2^18-node 20 x 20 bounding workload (seed 1), as the
    benchmark launches it, against the oracle node by node."""
    import torch
    p, _, rec = inputs.pool_workload(20, 20, 1, 2**18)
    inst = F.fsp_create_instance(p)
    got = F.fsp_bound_pool(inst, torch.from_numpy(rec).cuda()).cpu().numpy()
    F.fsp_check_status(inst)
    want = oracle.bound_pool(p, rec)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
