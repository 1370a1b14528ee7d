"""The seeded input generators (CPU): the counter-based generator against its
published outputs, and the images' determinism and statistics."""

import numpy as np

import synth


def test_splitmix64_published_outputs():
    # SplitMix64 (Steele, Lea and Flood, 2014) seeded with 0: its first three
    # outputs are e220a8397b1dcdaf, 6e789e6aa1b965f4, 06c45d188009454f
    z = synth.splitmix64(0, [0, 1, 2])
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform01_range_and_determinism():
    a = synth.uniform01(7, 3, 100000)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.01 and abs(a.var() - 1.0 / 12.0) < 0.005
    assert np.array_equal(a, synth.uniform01(7, 3, 100000))
    assert np.array_equal(a[10:20], synth.uniform01(7, 3, 10, offset=10))
    assert not np.array_equal(a[:100], synth.uniform01(7, 4, 100))
