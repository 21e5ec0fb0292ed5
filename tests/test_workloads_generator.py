"""The seeded input generator shared by the oracle and the library path:
SplitMix64 (Steele, Lea and Flood, 2014) pinned to its published first
outputs, its counter-based offsets, and the distributions built on it."""
import numpy as np

import workloads as wk


def test_splitmix64_matches_published_outputs():
    # the widely published first outputs of SplitMix64 for seeds 0 and 1234567
    assert [int(x) for x in wk.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in wk.splitmix64(1234567, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_splitmix64_offsets_continue_the_stream():
    whole = wk.splitmix64(42, 1000)
    assert np.array_equal(wk.splitmix64(42, 400, offset=600), whole[600:])
    assert np.array_equal(wk.splitmix64(42, 10), whole[:10])


def test_uniform_and_normal_distributions():
    u = wk.uniform(5, 200000, 0.0, 1.0)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12) < 2e-3
    v = wk.uniform(5, 1000, -1.0, 1.0)
    assert np.array_equal(v, -1.0 + 2.0 * u[:1000])
    z = wk.normal(6, 200001)
    assert z.size == 200001 and np.all(np.isfinite(z))
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1e-2
    # the fraction within one standard deviation, about 0.6827
    assert abs(np.mean(np.abs(z) < 1.0) - 0.6827) < 5e-3
