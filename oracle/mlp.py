"""Oracle of the learned pair-ordering network: node features, labels, and the
MLP's forward and backward passes in float64 with numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py).  The network is not in the
paper: it orders the two-machine bounds of a node so the one most likely to
reach the incumbent is evaluated first.  The kernels store some values in
bfloat16 (the inputs and weights they multiply, the hidden activations and
the back-propagated errors fed to the next product); this oracle rounds at
exactly those points with `bf16` below and computes everything else in
float64, so the two differ only by float32-vs-float64 accumulation.

Features of a node (prefix perm[:d]): C_k / T for every machine (release
times), S_k / T (remaining work), d / n, with T = total processing time / m;
float32, correctly rounded divisions.  Label: the first machine pair (k-major
numbering) whose two-machine bound equals the largest one.

Network: x (2m+1) -> relu(x W1 + b1) (H) -> relu(. W2 + b2) (H) -> . W3 + b3
(P = m(m-1)/2 scores); loss = mean cross-entropy of softmax(scores) against
the label.
"""
from __future__ import annotations

import numpy as np

import oracle


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(p, perm, d):
    """(x float32 [2m+1], label int) of one node."""
    p = np.asarray(p, dtype=np.int32)
    n, m = p.shape
    T = np.float32(np.float32(int(p.sum())) / np.float32(m))
    C = oracle.release_times(p, perm, d).astype(np.float32)
    S = p[np.asarray(perm[d:], dtype=np.int64)].sum(axis=0).astype(np.float32) if d < n else np.zeros(m, np.float32)
    x = np.concatenate([C / T, S / T, [np.float32(d) / np.float32(n)]]).astype(np.float32)
    _, _, pv = oracle.lb_parts(p, perm, d)
    return x, int(np.argmax(pv))


def _same(x):
    return np.asarray(x, dtype=np.float64)


def forward(params, X, rnd=bf16):
    """params: dict W1 [F,H], b1 [H], W2 [H,H], b2 [H], W3 [H,P], b3 [P] (float64
    values already representable in bf16 for the W's).  rnd: the rounding
    applied where the kernels store bf16 (`_same` switches it off).
    Returns the activations."""
    Xb = rnd(X)
    Z1 = Xb @ params["W1"] + params["b1"]
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = H1 @ params["W2"] + params["b2"]
    H2 = rnd(np.maximum(Z2, 0.0))
    L = H2 @ params["W3"] + params["b3"]
    return {"Xb": Xb, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2, "L": L}


def loss(params, X, y, rnd=bf16):
    a = forward(params, X, rnd)
    L = a["L"]
    Lm = L - L.max(axis=1, keepdims=True)
    lse = np.log(np.exp(Lm).sum(axis=1))
    return float(np.mean(lse - Lm[np.arange(X.shape[0]), y]))


def loss_and_grads(params, X, y, rnd=bf16):
    """Mean cross-entropy and its gradients for every parameter."""
    bf16 = rnd  # noqa: F811 -- the rounding points below follow the kernels
    a = forward(params, X, rnd)
    B = X.shape[0]
    L = a["L"]
    Lm = L - L.max(axis=1, keepdims=True)
    Pr = np.exp(Lm)
    Pr /= Pr.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(Pr[np.arange(B), y])))
    dL = Pr.copy()
    dL[np.arange(B), y] -= 1.0
    dL /= B
    g = {"W3": a["H2"].T @ bf16(dL), "b3": dL.sum(axis=0)}
    dH2 = bf16(dL) @ params["W3"].T
    dZ2 = dH2 * (a["H2"] > 0)
    g["W2"] = a["H1"].T @ bf16(dZ2)
    g["b2"] = dZ2.sum(axis=0)
    dH1 = bf16(dZ2) @ params["W2"].T
    dZ1 = dH1 * (a["H1"] > 0)
    g["W1"] = a["Xb"].T @ bf16(dZ1)
    g["b1"] = dZ1.sum(axis=0)
    return loss, g
