"""The seeded input generator: published SplitMix64 output, determinism, ranges."""
import numpy as np

from paper_2501_03245_gb300 import synth


def test_splitmix64_published_first_output():
    # SplitMix64 seeded with 0: first output is mix64(0x9E3779B97F4A7C15).
    assert int(synth._mix64(synth.GAMMA)) == 0xE220A8397B1DCDAF


def test_uniform_limbs_range_and_determinism():
    hi = (1 << 255) + 12345
    a = synth.uniform_limbs(42, 1, 5000, hi, lo=7)
    b = synth.uniform_limbs(42, 1, 5000, hi, lo=7)
    assert np.array_equal(a, b)
    vals = synth.limbs_to_ints(a)
    assert all(7 <= v < hi for v in vals)
    assert max(vals) > hi // 2  # uses the whole range
    c = synth.uniform_limbs(43, 1, 10, hi)
    assert not np.array_equal(a[:10], c)


def test_byte_conversions():
    x = synth.uniform_limbs(1, 2, 20, 1 << 256)
    be = synth.limbs_to_be32(x)
    assert np.array_equal(synth.be32_to_limbs(be), x)
    for i in range(20):
        assert int.from_bytes(bytes(be[i]), "big") == synth.limbs_to_int(x[i])


def test_ragged_sizes():
    s = synth.ragged_sizes(0x6ECC0003, 256)
    assert s.shape == (256,) and s.min() >= 1024 and s.max() < 2**18
    assert np.array_equal(s, synth.ragged_sizes(0x6ECC0003, 256))


def test_partial_shuffle_distinct():
    idx = synth.partial_shuffle(5, 4, 1000, 300)
    assert len(set(idx.tolist())) == 300 and idx.min() >= 0 and idx.max() < 1000
