"""The seeded input recipes produce what they claim (shapes, ranges, achieved
condition numbers, segment totals).  No GPU needed."""
import numpy as np
import pytest

import oracle
import workloads


def test_uniform_ranges_and_determinism():
    a = workloads.uniform_f32(1 << 16, seed=0)
    b = workloads.uniform_f32(1 << 16, seed=0)
    assert a.dtype == np.float32 and np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() <= 1.0
    i = workloads.uniform_i32(1 << 16, seed=0)
    assert i.dtype == np.int32 and i.min() == -1000 and i.max() == 1000


@pytest.mark.parametrize("cond", [1e4, 1e5, 1e6, 1e7, 1e8])
def test_cancelling_condition_numbers(cond):
    x = workloads.cancelling_f32(1 << 18, cond=cond, seed=0)
    s = abs(oracle.to_float(oracle.exact_f32(x)))
    c = oracle.sum_abs_f32(x) / s
    # heavy-tailed magnitudes make the realised cond scatter around the target
    assert cond / 30 <= c <= cond * 30, c


def test_segment_offsets_recipe():
    off = workloads.segment_offsets(10_000, 1 << 28, seed=0)
    lens = np.diff(off)
    assert off[0] == 0 and lens.min() >= 1 and lens.max() <= 1 << 24
    assert abs(int(off[-1]) - (1 << 28)) <= 0.01 * (1 << 28)
    assert 2000 < np.median(lens) < 8000


def test_fp8_and_bf16_encoding_shapes():
    x = workloads.lognormal_f32(1000, seed=1)
    codes, deq = workloads.to_e4m3_codes(x)
    assert codes.dtype == np.uint8 and codes.shape == x.shape
    assert not np.any((codes & 0x7F) == 0x7F)     # no NaN codes
    bits = workloads.to_bf16_bits(x)
    assert bits.dtype == np.uint16 and bits.shape == x.shape
