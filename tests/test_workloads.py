"""The seeded input generator (CPU only)."""
import numpy as np
import pytest

import workloads as W


def test_splitmix64_published_sequence():
    # SplitMix64 from state 0: the first outputs of the published generator
    # (Steele, Lea and Flood 2014), as also used to seed xoshiro generators.
    got = W.words(0, 0, 0, 3)
    assert [hex(int(v)) for v in got] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4",
                                          "0x6c45d188009454f"]


def test_counter_based_slices():
    full = W.words(5, 17, 0, 1000)
    assert np.array_equal(full[300:400], W.words(5, 17, 300, 100))


@pytest.mark.parametrize("dtype", W.DTYPES)
@pytest.mark.parametrize("dist", ["uniform", "zipf", "normal", "distinct8", "sorted", "reverse"])
def test_deterministic_and_typed(dtype, dist):
    a = W.make(dist, dtype, 5000, seed=3)
    b = W.make(dist, dtype, 5000, seed=3)
    assert a.dtype == (np.dtype(np.uint16) if dtype == "bfloat16" else np.dtype(dtype)) and a.size == 5000
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_distribution_shapes():
    assert np.unique(W.make("distinct8", "int64", 10000)).size == 8
    z = W.make("zipf", "uint32", 200000)
    vals, counts = np.unique(z, return_counts=True)
    assert vals.size > 1000 and counts.max() / z.size > 0.1  # heavy head, long tail
    e = W.make("float_edge", "float32", 200000).view(np.uint32)
    f = e.view(np.float32)
    assert 0.03 < np.isnan(f).mean() < 0.05
    assert 0.015 < np.isinf(f).mean() < 0.025
    sub = ((e & 0x7F800000) == 0) & ((e & 0x7FFFFF) != 0)
    assert 0.015 < sub.mean() < 0.025
    s = W.make("sorted", "int32", 1000)
    assert np.all(s[:-1] <= s[1:])


def test_segment_sizes_log_uniform():
    s = W.segment_sizes(0, 20000, 20)
    assert s.min() >= 1 and s.max() <= 1 << 20
    assert abs(np.log2(s).mean() - 10) < 0.3


def test_bf16_inputs():
    """bfloat16 comes as uint16 patterns: normal values round to nearest even
    from binary32, the edge mix has its NaN / inf / subnormal shares."""
    x = W.make("normal", "bfloat16", 100000, seed=1)
    f = (x.astype(np.uint32) << 16).view(np.float32)
    assert np.all(np.isfinite(f)) and 600 < np.std(f) < 1400
    e = W.make("float_edge", "bfloat16", 200000, seed=2).astype(np.uint32)
    exp, man = (e >> 7) & 0xFF, e & 0x7F
    assert 0.03 < ((exp == 0xFF) & (man != 0)).mean() < 0.05
    assert 0.015 < ((exp == 0xFF) & (man == 0)).mean() < 0.025
    assert 0.015 < ((exp == 0) & (man != 0)).mean() < 0.025
    assert W._bf16_bits(np.array([1.0, -2.5, 1.00390625, 1.01171875])).tolist() == [0x3F80, 0xC020, 0x3F80, 0x3F82]
