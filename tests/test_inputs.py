"""The seeded input generator shared by the oracle and the GPU tests: its
stream is SplitMix64 as published (reference outputs of the generator's
definition for seeds 0 and 1234567), and the recipes give values in range."""
import numpy as np

from paper_1206_4973_gb300 import inputs


def test_splitmix64_reference_outputs():
    assert [int(x) for x in inputs.SplitMix64(0).take(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in inputs.SplitMix64(1234567).take(2)] == [6457827717110365317, 3203168211198807973]


def test_stream_is_counter_based():
    a = inputs.SplitMix64(99)
    first = a.take(5)
    b = inputs.SplitMix64(99)
    assert np.array_equal(np.concatenate([b.take(2), b.take(3)]), first)


def test_instances_and_pools_are_in_range():
    p = inputs.instance(20, 20, 1)
    assert p.shape == (20, 20) and p.dtype == np.int32 and p.min() >= 1 and p.max() <= 99
    rec = inputs.random_prefix_pool(20, 500, inputs.SplitMix64(3))
    assert rec.shape == (500, 32)
    assert all(sorted(r[:20]) == list(range(20)) for r in rec)
    assert rec[:, 20].min() >= 1 and rec[:, 20].max() <= 19 and not rec[:, 21:].any()
