"""Per-element error bounds for the network's gradients (test helper, no
GPU): how far a gradient computed by the kernels (bf16 operands, fp32
accumulation) may lie from the fp64 oracle's (oracle/mlp.py), element by
element."""
import numpy as np

from oracle import mlp as om

ULP = 2.0**-7    # one bf16 ulp, relative: the neighbour a rounding can land on instead


def gamma(k):
    """fp32 accumulation of k terms (2 k u, u = 2^-24: covers round-to-nearest
    and truncating adders), relative to the sum of |terms|."""
    return 2.0 * k * 2.0**-24


def bf16_boundary_distance(x):
    """Distance from each value to the nearest bf16 rounding midpoint: a
    value closer to a midpoint than its own error bound may round to the
    other neighbour on the GPU; any other value rounds identically."""
    x = np.asarray(x, np.float64)
    r = om.bf16(x).astype(np.float32)
    hi = r.view(np.uint32) >> np.uint32(16)
    up = ((hi + np.uint32(1)) << np.uint32(16)).view(np.float32).astype(np.float64)
    dn = ((np.maximum(hi, 1) - np.uint32(1)) << np.uint32(16)).view(np.float32).astype(np.float64)
    rr = r.astype(np.float64)
    d = np.minimum(np.abs(x - (rr + up) / 2), np.abs(x - (rr + dn) / 2))
    return np.where((hi & np.uint32(0x7FFF)) == 0, 0.0, d)


def rounded_error(x, ex):
    """Error bound of bf16(x) on the GPU given |x_gpu - x| <= ex: none unless
    x is within ex of a rounding midpoint, then one ulp plus ex."""
    risk = bf16_boundary_distance(x) <= ex
    return np.where(risk, ULP * np.abs(x) + ex, 0.0)


def gradient_bounds(prm, X, y):
    """Per-element bounds on |GPU gradient - oracle gradient|.  The two sides
    multiply the same bf16 weights and inputs; they differ by fp32 against
    fp64 accumulation (gamma(k) times the sum of |terms|), and by a bf16
    rounding that lands on the other neighbour, which can only happen where
    the oracle's value lies within its error bound of a rounding midpoint
    (rounded_error), or by a ReLU that can only flip where the
    pre-activation lies within its error bound of zero.  Each bound is
    propagated through the layers as the kernels compute them."""
    a = om.forward(prm, X)
    B = X.shape[0]
    aW1, aW2, aW3 = np.abs(prm["W1"]), np.abs(prm["W2"]), np.abs(prm["W3"])
    aX = np.abs(a["Xb"])
    # forward: Z = H W + b in fp32, then bf16(relu(Z))
    eZ1 = gamma(aW1.shape[0] + 1) * (aX @ aW1 + np.abs(prm["b1"]))
    eH1 = np.where(np.abs(a["Z1"]) <= eZ1, np.abs(a["Z1"]) + eZ1, rounded_error(np.maximum(a["Z1"], 0), eZ1))
    mH1 = np.abs(a["H1"]) + eH1
    eZ2 = eH1 @ aW2 + gamma(aW2.shape[0] + 1) * (mH1 @ aW2 + np.abs(prm["b2"]))
    eH2 = np.where(np.abs(a["Z2"]) <= eZ2, np.abs(a["Z2"]) + eZ2, rounded_error(np.maximum(a["Z2"], 0), eZ2))
    mH2 = np.abs(a["H2"]) + eH2
    eL = eH2 @ aW3 + gamma(aW3.shape[0] + 1) * (mH2 @ aW3 + np.abs(prm["b3"]))
    # softmax cross-entropy in fp32: a probability moves by at most 2 max|dL| relative
    L = a["L"]
    Pr = np.exp(L - L.max(axis=1, keepdims=True))
    Pr /= Pr.sum(axis=1, keepdims=True)
    dL = Pr.copy()
    dL[np.arange(B), y] -= 1.0
    dL /= B
    edL = (2.0 * eL.max(axis=1, keepdims=True) + 2.0**-20) * Pr / B + 2.0**-22 * np.abs(dL)
    edLb = rounded_error(dL, edL)
    mdLb = np.abs(om.bf16(dL)) + edLb
    gb = gamma(B)
    out = {"W3": eH2.T @ mdLb + mH2.T @ edLb + gb * (mH2.T @ mdLb),
           "b3": edL.sum(axis=0) + gb * np.abs(dL).sum(axis=0)}
    # layer 2: dZ2 = (bf16(dL) W3^T) masked by H2 > 0, rounded to bf16 for the products
    dH2 = om.bf16(dL) @ prm["W3"].T
    edH2 = edLb @ aW3.T + gamma(aW3.shape[1]) * (mdLb @ aW3.T)
    flip2 = np.abs(a["Z2"]) <= eZ2
    dZ2 = np.where(a["H2"] > 0, dH2, 0.0)
    edZ2 = np.where(flip2, np.abs(dH2) + edH2, np.where(a["H2"] > 0, edH2, 0.0))
    edZ2b = rounded_error(dZ2, edZ2)
    mdZ2b = np.abs(om.bf16(dZ2)) + edZ2b
    out["W2"] = eH1.T @ mdZ2b + mH1.T @ edZ2b + gb * (mH1.T @ mdZ2b)
    out["b2"] = edZ2.sum(axis=0) + gb * (np.abs(dZ2) + edZ2).sum(axis=0)
    # layer 1
    dH1 = om.bf16(dZ2) @ prm["W2"].T
    edH1 = edZ2b @ aW2.T + gamma(aW2.shape[1]) * (mdZ2b @ aW2.T)
    flip1 = np.abs(a["Z1"]) <= eZ1
    dZ1 = np.where(a["H1"] > 0, dH1, 0.0)
    edZ1 = np.where(flip1, np.abs(dH1) + edH1, np.where(a["H1"] > 0, edH1, 0.0))
    edZ1b = rounded_error(dZ1, edZ1)
    mdZ1b = np.abs(om.bf16(dZ1)) + edZ1b
    out["W1"] = aX.T @ edZ1b + gb * (aX.T @ mdZ1b)
    out["b1"] = edZ1.sum(axis=0) + gb * (np.abs(dZ1) + edZ1).sum(axis=0)
    return out
