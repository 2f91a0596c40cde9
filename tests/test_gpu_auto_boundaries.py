"""SR_AUTO at the edges of its size regimes: one element below, at and
above every byte size where the table changes shape (1, 4, 8, 16, 32 and
64 MiB), for every input type, plain and compensated, at an aligned and a
misaligned start.  The values are small integers (|v| <= 4), exact in BF16
and E4M3, whose every partial sum stays far below 2^24 in magnitude, so each
result must equal the oracle's exact integer sum bit for bit whatever the
launch shape."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu
MIB = 1 << 20
BOUNDARIES = [1 * MIB, 4 * MIB, 8 * MIB, 16 * MIB, 32 * MIB, 64 * MIB]


@pytest.fixture(scope="module")
def values():
    n = 64 * MIB + 16
    v = workloads.uniform_i32(n, seed=77, lo=-4, hi=4)
    return v, torch.from_numpy(v).cuda()


def _input(vd, dtype, sr, n, off):
    conv = {sr.F32: lambda t: t.float(), sr.I32: lambda t: t,
            sr.BF16: lambda t: t.float().to(torch.bfloat16),
            sr.FP8E4M3: lambda t: t.float().to(torch.float8_e4m3fn).view(torch.uint8)}[dtype]
    src = conv(vd[:n + off])
    buf = torch.zeros(src.numel() + 16, dtype=src.dtype, device="cuda")
    buf[:src.numel()] = src
    return buf[off:off + n]


@pytest.mark.parametrize("dtype_name,comp", [("F32", 0), ("F32", 1), ("I32", 0), ("BF16", 0), ("BF16", 1),
                                             ("FP8E4M3", 0), ("FP8E4M3", 1)])
@pytest.mark.parametrize("boundary", BOUNDARIES)
def test_auto_regime_boundaries_exact(sr, values, dtype_name, comp, boundary):
    v, vd = values
    dtype = getattr(sr, dtype_name)
    eb = {sr.F32: 4, sr.I32: 4, sr.BF16: 2, sr.FP8E4M3: 1}[dtype]
    variant = sr.AUTO | (sr.F_KAHAN if comp else 0)
    out_dt = torch.int64 if dtype == sr.I32 else torch.float32
    for n in (boundary // eb - 1, boundary // eb, boundary // eb + 1):
        if n > v.size - 16:
            continue
        for off in (0, 1):
            x = _input(vd, dtype, sr, n, off)
            want = oracle.sum_i32(v[off:off + n])
            out = torch.full((1,), -12345, dtype=out_dt, device="cuda")
            sr.check(sr.reduce_sum_ptr(x.data_ptr(), n, dtype, out.data_ptr(), sr.make_config(variant), 0))
            torch.cuda.synchronize()
            got = out.item()
            assert got == want, (dtype_name, comp, n, off, got, want, sr.plan(n, dtype, sr.make_config(variant)).as_dict())
