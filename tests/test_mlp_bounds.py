"""The per-element gradient bounds of tests/mlp_bounds.py are not vacuous:
a single gradient element moved by a few percent of the tensor's largest
entry (planted in the oracle's output, on the CPU) breaks them, where a
relative-norm comparison of the whole tensor would still pass.  No GPU."""
import numpy as np
import pytest

import mlp_bounds as mb
from oracle import mlp as om


def network(seed, F_=41, H=128, P=190):
    rng = np.random.default_rng(seed)
    return {"W1": om.bf16(rng.normal(0, 0.2, (F_, H))), "b1": np.zeros(H),
            "W2": om.bf16(rng.normal(0, 0.1, (H, H))), "b2": np.zeros(H),
            "W3": om.bf16(rng.normal(0, 0.1, (H, P))), "b3": np.zeros(P)}, rng


@pytest.mark.parametrize("kind,key", [("dense", "W2"), ("dense", "W3"), ("onehot", "W1"), ("onehot", "b2")])
def test_a_planted_wrong_element_is_caught(kind, key):
    prm, rng = network(5)
    B, F_, P = 64, 41, 190
    if kind == "dense":
        X = rng.uniform(0, 2, size=(B, F_)).astype(np.float32)
    else:
        X = np.zeros((B, F_), np.float32)
        X[np.arange(B), rng.integers(0, F_, B)] = 1.0
    y = rng.integers(0, P, size=B).astype(np.int32)
    _, g0 = om.loss_and_grads(prm, X, y)
    tol = mb.gradient_bounds(prm, X, y)
    assert all(np.all(tol[k] >= 0) for k in g0)
    bad = g0[key].copy()
    i = np.unravel_index(np.argmax(np.abs(g0[key]) - 50 * tol[key]), bad.shape)
    bad[i] += 0.03 * np.abs(g0[key]).max()
    assert np.linalg.norm(bad - g0[key]) / np.linalg.norm(g0[key]) <= 2.0**-5  # a norm test passes
    assert not np.all(np.abs(bad - g0[key]) <= tol[key])


def test_identical_values_far_from_rounding_midpoints_have_no_rounding_error():
    x = np.array([1.0, 1.5, -3.0, 0.75])  # bf16 values themselves: half an ulp from any midpoint
    d = mb.bf16_boundary_distance(x)
    assert np.all(d > 0)
    assert np.all(mb.rounded_error(x, d / 2) == 0)
    assert np.all(mb.rounded_error(x, d * 2) > 0)
