"""Precision path: BF16 / FP8-E4M3 inputs accumulated in FP32, two-sum
compensated accumulation (SR_F_KAHAN) and the binary64 cross-unit combine
(SR_F_FP64_COMBINE), against the exact sum of the decoded inputs.

Gates (u = 2^-24):
  plain FP32 tree, random-sign data : |err| <= 4 eps32 sum|x|          (stated gate)
  compensated, any data             : |err| <= (2u + n u^2) sum|x|     (Kahan's bound)
  compensated, cond <= 10           : |err| / |S| <= 1e-6              (stated gate)
  compensated + FP64 combine,
  cancelling data up to cond 1e8    : |err| / |S| <= 1e-6
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _dev(arr, torch_dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    return t.view(torch_dtype) if torch_dtype is not None else t


def _bf16(bits):
    return _dev(bits.view(np.int16), torch.bfloat16)


def _run(sr, x, variant, **cfg):
    return float(sr.reduce_sum(x, config=sr.make_config(variant, **cfg)).item())


def _kahan_bound(n, sabs):
    return (2 * U + n * U * U) * sabs


@pytest.mark.parametrize("stage", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("flags", [0, 0x100, 0x300, 0x400, 0x500])
def test_bf16_parity(sr, stage, flags):
    for n in [0, 1, 7, 33, 1029, (1 << 18) + 3]:
        x = workloads.lognormal_f32(n, seed=n + 1, sigma=4.0)
        bits = workloads.to_bf16_bits(x)
        exact = oracle.to_float(oracle.exact_bf16(bits))
        dec = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
        sabs = oracle.sum_abs_f32(dec)
        for off in (0, 1, 3):
            buf = np.zeros(n + off, np.uint16)
            buf[off:] = bits
            xd = _bf16(buf)[off:]
            got = _run(sr, xd, stage | flags)
            err = abs(got - exact)
            if flags & 0x100:
                assert err <= _kahan_bound(n, sabs) + 1e-300, (n, off, got, exact)
            else:
                assert err <= oracle.stated_fp32_bound(sabs), (n, off, got, exact)


@pytest.mark.parametrize("stage", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("flags", [0, 0x100, 0x300, 0x400])
def test_fp8_parity(sr, stage, flags):
    for n in [0, 1, 15, 17, 1031, (1 << 18) + 9]:
        x = workloads.lognormal_f32(n, seed=n + 2, sigma=2.0)
        codes, deq = workloads.to_e4m3_codes(x)
        exact = oracle.to_float(oracle.exact_e4m3(codes, deq))
        sabs = oracle.sum_e4m3(codes & 0x7F, deq)
        for off in (0, 1, 5, 15):
            buf = np.zeros(n + off, np.uint8)
            buf[off:] = codes
            xd = _dev(buf)[off:]
            got = _run(sr, xd, stage | flags, scale=deq)
            err = abs(got - exact)
            if flags & 0x100:
                assert err <= _kahan_bound(n, sabs) * 1.01 + 1e-300, (n, off, got, exact)
            else:
                assert err <= oracle.stated_fp32_bound(sabs), (n, off, got, exact)


def test_fp8_scale_applied_once(sr):
    codes = np.array([0x38] * 1000, np.uint8)        # 1000 x 1.0
    got = _run(sr, _dev(codes), sr.LAST_BLOCK, scale=0.25)
    assert got == 250.0


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_compensated_relative_error_well_conditioned(sr, dtype):
    """cond = sum|x| / |S| = 1 (positive lognormal data): relative error <= 1e-6
    with compensation; the plain tree is reported alongside."""
    n = (1 << 22) + 5
    x = np.abs(workloads.lognormal_f32(n, seed=7, sigma=1.0))
    if dtype == "f32":
        xd, exact, kw = _dev(x), oracle.exact_f32(x), {}
    elif dtype == "bf16":
        bits = workloads.to_bf16_bits(x)
        xd, exact, kw = _bf16(bits), oracle.exact_bf16(bits), {}
    else:
        codes, deq = workloads.to_e4m3_codes(x)
        xd, exact, kw = _dev(codes), oracle.exact_e4m3(codes, deq), {"scale": deq}
    S = oracle.to_float(exact)
    for stage in (sr.TWO_KERNEL, sr.LAST_BLOCK, sr.GRID_SYNC, sr.ATOMIC):
        for flags in (sr.F_KAHAN, sr.F_KAHAN | sr.F_FP64_COMBINE, sr.F_KAHAN | sr.F_BULK):
            got = _run(sr, xd, stage | flags, **kw)
            assert abs(got - S) / abs(S) <= 1e-6, (dtype, stage, flags, got, S)


@pytest.mark.parametrize("cond", [1e4, 1e6, 1e8])
def test_fp64_combine_on_cancelling_sums(sr, cond):
    n = 1 << 22
    x = workloads.cancelling_f32(n, cond=cond, seed=0)
    exact = oracle.exact_f32(x)
    S = oracle.to_float(exact)
    sabs = oracle.sum_abs_f32(x)
    xd = _dev(x)
    for stage in (sr.TWO_KERNEL, sr.LAST_BLOCK, sr.GRID_SYNC):
        got = _run(sr, xd, stage | sr.F_KAHAN | sr.F_FP64_COMBINE)
        assert abs(got - S) <= _kahan_bound(n, sabs)
        assert abs(got - S) / abs(S) <= 1e-6, (cond, stage, got, S)
        got_k = _run(sr, xd, stage | sr.F_KAHAN)
        assert abs(got_k - S) <= _kahan_bound(n, sabs)


def test_fp64_combine_output_is_double(sr):
    x = _dev(workloads.uniform_f32(1 << 16, seed=3))
    out = sr.reduce_sum(x, variant=sr.LAST_BLOCK | sr.F_FP64_COMBINE)
    assert out.dtype == torch.float64


@pytest.mark.slow
def test_full_size_precision_workloads(sr):
    """The precision workload at its full size (n = 2^28): lognormal(0, 4)
    magnitudes with random signs in FP32, BF16 and FP8, plain / compensated /
    compensated + FP64 combine (SR_AUTO launch shapes), and cancelling FP32
    pairs at cond ~1e8 — every result inside its gate."""
    n = 1 << 28
    x = workloads.lognormal_f32(n, seed=0, sigma=4.0)
    cases = [("f32", _dev(x), oracle.exact_f32(x), oracle.sum_abs_f32(x), {})]
    bits = workloads.to_bf16_bits(x)
    dec = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
    cases.append(("bf16", _bf16(bits), oracle.exact_bf16(bits), oracle.sum_abs_f32(dec), {}))
    del dec
    codes, deq = workloads.to_e4m3_codes(x)
    cases.append(("fp8", _dev(codes), oracle.exact_e4m3(codes, deq), oracle.sum_e4m3(codes & 0x7F, deq),
                  {"scale": deq}))
    del x
    for name, xd, exact, sabs, kw in cases:
        S = oracle.to_float(exact)
        got = _run(sr, xd, sr.AUTO, **kw)
        assert abs(got - S) <= oracle.stated_fp32_bound(sabs), name
        for flags in (sr.F_KAHAN, sr.F_KAHAN | sr.F_FP64_COMBINE):
            got = _run(sr, xd, sr.AUTO | flags, **kw)
            assert abs(got - S) <= _kahan_bound(n, sabs), (name, flags)
            assert abs(got - S) / abs(S) <= 1e-6, (name, flags, got, S)   # cond ~ 43 here
        del xd
        torch.cuda.empty_cache()
    xc = workloads.cancelling_f32(n, cond=1e8, seed=0)
    S = oracle.to_float(oracle.exact_f32(xc))
    got = _run(sr, _dev(xc), sr.AUTO | sr.F_KAHAN | sr.F_FP64_COMBINE)
    assert abs(got - S) / abs(S) <= 1e-6, (got, S)


def test_fp64_auto_combine(sr):
    """SR_F_FP64_AUTO: binary64 only in the cross-unit combine and only when the
    pair combine's bound is not met — identical to the compensated result on
    well-conditioned data, within 1e-6 relative on cond ~1e8 data."""
    x = np.abs(workloads.lognormal_f32((1 << 22) + 3, seed=7, sigma=1.0))
    xd = _dev(x)
    for stage in (sr.TWO_KERNEL, sr.LAST_BLOCK, sr.GRID_SYNC):
        a = _run(sr, xd, stage | sr.F_KAHAN)
        b = _run(sr, xd, stage | sr.F_FP64_AUTO)
        assert a == b
    n = 1 << 22
    xc = workloads.cancelling_f32(n, cond=1e8, seed=0)
    S = oracle.to_float(oracle.exact_f32(xc))
    xd = _dev(xc)
    for stage in (sr.TWO_KERNEL, sr.LAST_BLOCK, sr.GRID_SYNC):
        out = sr.reduce_sum(xd, variant=stage | sr.F_FP64_AUTO)
        assert out.dtype == torch.float32
        assert abs(float(out.item()) - S) / abs(S) <= 1e-6
