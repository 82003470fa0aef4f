"""The shared input generator: counter-based SplitMix64, host and torch paths."""
import numpy as np
import torch

import synth


def test_known_splitmix64_outputs():
    # SplitMix64 seeded with 0: the first outputs of the published generator.
    assert synth.splitmix64_scalar(0, 0) == 0xE220A8397B1DCDAF
    assert synth.splitmix64_scalar(0, 1) == 0x6E789E6AA1B965F4
    assert synth.splitmix64_scalar(0, 2) == 0x06C45D188009454F


def test_numpy_matches_scalar():
    for seed in (0, 0xC1A2, (1 << 64) - 5):
        vals = synth.uniform_np(seed, 100, 50)
        for k in range(50):
            z = synth.splitmix64_scalar(seed, 100 + k)
            assert vals[k] == 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0


def test_torch_matches_numpy_bitwise():
    a = synth.uniform_np(0xC1A3, 12345, 100000)
    b = synth.uniform_torch(0xC1A3, 12345, 100000, "cpu", chunk=4096).numpy()
    np.testing.assert_array_equal(a, b)


def test_range_and_moments():
    v = synth.uniform_np(0xC1A1, 0, 1 << 16)
    assert v.min() >= -1.0 and v.max() < 1.0
    assert abs(v.mean()) < 0.01 and abs(v.var() - 1.0 / 3.0) < 0.01


def test_uneven_sizes_ranges():
    n, t = synth.uneven_sizes(0xC1A4, 10000)
    assert n.min() >= 2 and n.max() <= 64 and t.min() >= 16 and t.max() <= 128
    # log-uniform: about as many instances in [2,8) as in [8,32)
    a = np.sum((n >= 2) & (n < 8))
    b = np.sum((n >= 8) & (n < 32))
    assert 0.7 < a / b < 1.4


def test_layout_roundtrip():
    x = synth.uniform_np(1, 0, 2 * 3 * 4).reshape(2, 3, 4)
    for lay in range(6):
        np.testing.assert_array_equal(synth.from_layout(synth.to_layout(x, lay).ravel(), lay, x.shape), x)
