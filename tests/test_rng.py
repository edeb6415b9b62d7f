"""Pins of the seeded generator: SplitMix64's published first outputs for
state 0 (Vigna's reference implementation) and the moments of Box-Muller."""
import numpy as np

from problems import rng


def test_splitmix64_reference_values():
    z = rng.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_offsets_are_consistent():
    a = rng.splitmix64(7, 10)
    b = rng.splitmix64(7, 5, offset=5)
    assert np.array_equal(a[5:], b)


def test_uniform_and_normal_moments():
    u = rng.uniform(3, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    z = rng.normal(4, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2
    k = rng.integers(5, 100000, 32, 192)
    assert k.min() == 32 and k.max() == 192
