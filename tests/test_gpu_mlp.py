"""GPU parity of the learned-order network with its oracle (oracle/mlp.py):
features and labels exact, forward scores within bounds derived from bf16
rounding, every gradient element within its propagated bound
(tests/mlp_bounds.py), and training that lowers the loss."""
import numpy as np
import pytest

import mlp_bounds as mb
import oracle
from oracle import mlp as om
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


@pytest.mark.parametrize("n,m,seed,count", [(20, 20, 6, 700), (50, 20, 7, 300), (12, 5, 0, 500), (9, 3, 2, 200)])
def test_features_and_labels_match_oracle(F, n, m, seed, count):
    import torch
    p = inputs.instance(n, m, seed)
    rng = inputs.SplitMix64(seed + 1000)
    rec = inputs.random_prefix_pool(n, count, rng)
    rec[::5, n] = 0
    inst = F.fsp_create_instance(p)
    x, y = F.fsp_node_features(inst, torch.from_numpy(rec).cuda())
    x, y = x.cpu().numpy(), y.cpu().numpy()
    for t in range(count):
        xo, yo = om.features(p, rec[t, :n], rec[t, n])
        assert np.array_equal(x[t], xo), t
        assert y[t] == yo, t


def params_dict(mlp, flat):
    return {k: om.bf16(v) if k.startswith("W") else v.astype(np.float64) for k, v in mlp.split(flat).items()}


def product_bound(a, w):
    """|error| allowed in a @ w: two bf16 ulps (2^-7 relative) on each operand
    term, plus fp32 accumulation."""
    return 2.0**-7 * (np.abs(a) @ np.abs(w)) + 1e-5


@pytest.mark.parametrize("F_,H,P,B", [(41, 128, 190, 256), (11, 128, 10, 100), (101, 128, 190, 77)])
def test_forward_matches_oracle(F, F_, H, P, B):
    import torch
    mlp = F.Mlp(F_, H, P, seed=3)
    rng = np.random.default_rng(7)
    X = rng.uniform(0, 2, size=(B, F_)).astype(np.float32)
    got = mlp.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    prm = params_dict(mlp, mlp.get_params())
    a = om.forward(prm, X)
    tol = product_bound(a["H2"], prm["W3"])
    assert np.all(np.abs(got - a["L"]) <= tol), float(np.max(np.abs(got - a["L"]) - tol))


def net_inputs(kind, F_, B, P, seed):
    rng = np.random.default_rng(seed + 2)
    if kind == "dense":
        X = rng.uniform(0, 2, size=(B, F_)).astype(np.float32)
    else:  # one-hot rows: the first layer's pre-activations are single bf16 weights (exact)
        X = np.zeros((B, F_), np.float32)
        X[np.arange(B), rng.integers(0, F_, B)] = 1.0
    return X, rng.integers(0, P, size=B).astype(np.int32)


# median bound / largest |gradient| asserted per tensor: the tensors whose
# bound no rounding cascade widens (with one-hot inputs also the first layer)
TIGHT = {"dense": {"W3": 0.02, "b3": 0.02, "W2": 0.02},
         "onehot": {"W3": 0.02, "b3": 0.02, "W2": 0.02, "b2": 0.05, "W1": 0.05}}


@pytest.mark.parametrize("kind,F_,H,P,B,seed", [("dense", 41, 128, 190, 64, 11), ("dense", 11, 128, 10, 100, 12),
                                                ("dense", 101, 128, 190, 33, 14), ("onehot", 41, 128, 190, 64, 15)])
def test_gradients_match_oracle_elementwise(F, kind, F_, H, P, B, seed):
    """Every gradient element within its propagated bound
    (tests/mlp_bounds.py), and the bound is tight where no rounding cascade
    can widen it."""
    import torch
    mlp = F.Mlp(F_, H, P, seed=seed)
    X, y = net_inputs(kind, F_, B, P, seed)
    loss, g = mlp.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    g = mlp.split(g.cpu().numpy())
    prm = params_dict(mlp, mlp.get_params())
    loss0, g0 = om.loss_and_grads(prm, X, y)
    assert abs(loss - loss0) <= 1e-3 * max(1.0, abs(loss0))
    tol = mb.gradient_bounds(prm, X, y)
    for k in g0:
        diff = np.abs(g[k].astype(np.float64) - g0[k])
        assert np.all(diff <= tol[k]), (k, float(np.max(diff - tol[k])), np.unravel_index(np.argmax(diff - tol[k]),
                                                                                          diff.shape))
    for k, frac in TIGHT[kind].items():
        live = np.abs(g0[k]) > 0
        assert np.median(tol[k][live]) <= frac * np.abs(g0[k]).max(), (k, float(np.median(tol[k][live])))


def test_training_lowers_the_loss_on_solver_nodes(F):
    """Random 20 x 20 nodes, their features and labels, 200 Adam steps."""
    import torch
    n, m = 20, 20
    p = inputs.instance(n, m, 6)
    inst = F.fsp_create_instance(p)
    rec = inputs.random_prefix_pool(n, 8192, inputs.SplitMix64(66))
    x, y = F.fsp_node_features(inst, torch.from_numpy(rec).cuda())
    P = m * (m - 1) // 2
    mlp = F.Mlp(2 * m + 1, 128, P, seed=1)
    first = mlp.train_step(x[:1024], y[:1024], lr=2e-3)
    for it in range(200):
        s = (it * 1024) % 8192
        mlp.train_step(x[s:s + 1024], y[s:s + 1024], lr=2e-3)
    l_end, _ = mlp.loss_grad(x, y)
    assert l_end < first * 0.8, (first, l_end)
    # it beats the best constant prediction (the label frequencies): their entropy
    freq = np.bincount(y.cpu().numpy(), minlength=P) / len(y)
    entropy = -np.sum(freq[freq > 0] * np.log(freq[freq > 0]))
    assert l_end < entropy, (l_end, entropy)


@pytest.mark.parametrize("m,n,k", [(20, 20, 4), (10, 15, 8), (5, 12, 2), (20, 50, 1)])
def test_fused_pair_order_matches_oracle_scores(F, m, n, k):
    """The fused kernel's top-k pairs are the oracle's best-scored pairs, up to
    scores closer than the forward tolerance."""
    import torch
    P = m * (m - 1) // 2
    p = inputs.instance(n, m, 40 + m)
    inst = F.fsp_create_instance(p)
    rec = inputs.random_prefix_pool(n, 300, inputs.SplitMix64(77 + m))
    mlp = F.Mlp(2 * m + 1, 128, P, seed=m)
    top = F.fsp_pair_order(inst, mlp, torch.from_numpy(rec).cuda(), k=k).cpu().numpy()
    prm = params_dict(mlp, mlp.get_params())
    X = np.stack([om.features(p, rec[t, :n], rec[t, n])[0] for t in range(len(rec))])
    a = om.forward(prm, X)
    tol = product_bound(a["H2"], prm["W3"]) * 2 + 1e-4
    for t in range(len(rec)):
        sc = a["L"][t]
        assert len(set(top[t].tolist())) == k and top[t].max() < P
        kth = np.sort(sc)[::-1][k - 1]
        for j, q in enumerate(top[t]):
            assert sc[q] >= kth - tol[t].max(), (t, j, q)
        # best first
        assert np.all(np.diff(sc[top[t]]) <= tol[t].max())
