"""Seeded synthetic inputs for the flow-shop bounding path.

This module holds no arithmetic of the method: it only draws random numbers
and lays them out.  Both the CUDA path's tests/benchmarks and the CPU oracle
take their inputs from here.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  With state s0 = seed, the k-th output
(k = 0, 1, ...) is mix(s0 + (k + 1) * 0x9E3779B97F4A7C15) where
mix(z) = z ^ z>>30, * 0xBF58476D1CE4E5B9, ^ >>27, * 0x94D049BB133111EB, ^ >>31.
Being counter-based it vectorises over k.

Recipe (stand-in for the Taillard instances the paper uses, Sec. V-A, which
are not available here): processing times p[j][k] = 1 + (x >> 32) % 99 drawn
job-major; random permutations by Fisher-Yates with i from n-1 down to 1 and
j = (x >> 32) % (i + 1); node depths d = 1 + (x >> 32) % (n - 1).  The stream
order is: instance, then (pool workloads) one permutation for the UB, then per
node its permutation followed by its depth.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def node_stride(n: int) -> int:
    """Bytes per node record: perm[n], depth at byte n, zero pad to 16 bytes."""
    return (n + 1 + 15) // 16 * 16


class SplitMix64:
    """Counter-based SplitMix64 stream with a position cursor."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0

    def take(self, count: int) -> np.ndarray:
        k = np.arange(self.pos + 1, self.pos + 1 + count, dtype=np.uint64)
        self.pos += count
        with np.errstate(over="ignore"):
            z = self.seed + k * GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def take_hi(self, count: int) -> np.ndarray:
        """High 32 bits of the next `count` outputs (as uint64)."""
        return self.take(count) >> np.uint64(32)


def instance(n: int, m: int, seed: int, rng: SplitMix64 | None = None) -> np.ndarray:
    """p[n, m] int32, job-major, uniform in [1, 99]."""
    rng = rng if rng is not None else SplitMix64(seed)
    hi = rng.take_hi(n * m)
    return (np.uint64(1) + hi % np.uint64(99)).astype(np.int32).reshape(n, m)


def _fisher_yates(hi: np.ndarray, n: int) -> np.ndarray:
    """hi: [count, n-1] draws -> [count, n] permutations."""
    count = hi.shape[0]
    perms = np.tile(np.arange(n, dtype=np.uint8), (count, 1))
    rows = np.arange(count)
    for s, i in enumerate(range(n - 1, 0, -1)):
        j = (hi[:, s] % np.uint64(i + 1)).astype(np.int64)
        a = perms[:, i].copy()
        perms[:, i] = perms[rows, j]
        perms[rows, j] = a
    return perms


def permutation(n: int, rng: SplitMix64) -> np.ndarray:
    return _fisher_yates(rng.take_hi(n - 1).reshape(1, n - 1), n)[0]


def random_prefix_pool(n: int, count: int, rng: SplitMix64, max_depth: int | None = None) -> np.ndarray:
    """count node records: prefix of a random permutation, depth uniform in [1, n-1]."""
    if n < 2:
        raise ValueError("pool nodes need n >= 2")
    dmax = (n - 1) if max_depth is None else max_depth
    hi = rng.take_hi(count * n).reshape(count, n)
    perms = _fisher_yates(hi[:, : n - 1], n)
    depth = (np.uint64(1) + hi[:, n - 1] % np.uint64(dmax)).astype(np.uint8)
    rec = np.zeros((count, node_stride(n)), np.uint8)
    rec[:, :n] = perms
    rec[:, n] = depth
    return rec


def pool_workload(n: int, m: int, seed: int, count: int):
    """Bounding microbenchmark: (p, UB permutation, node records).

    The UB is the makespan of the returned permutation (computed by whoever
    consumes it); the nodes are prefixes of random permutations.
    """
    rng = SplitMix64(seed)
    p = instance(n, m, seed, rng)
    ub_perm = permutation(n, rng)
    nodes = random_prefix_pool(n, count, rng)
    return p, ub_perm, nodes


def batch_shapes(count: int = 256, first_seed: int = 100):
    """Mixed-shape batch: instance i has n = (12, 15, 20, 50)[i % 4],
    m = (5, 10)[(i // 4) % 2] and seed first_seed + i."""
    out = []
    for i in range(count):
        out.append(((12, 15, 20, 50)[i % 4], (5, 10)[(i // 4) % 2], first_seed + i))
    return out
