"""sr_reduce_sum_host (host input, host result) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [0, 1, 1000, (1 << 24) + 7, (1 << 26) + 5])
def test_host_entry_parity(sr, n):
    xf = workloads.uniform_f32(n, seed=3)
    xi = workloads.uniform_i32(n, seed=3)
    for arr, dt, pin in ((xf, sr.F32, True), (xi, sr.I32, True), (xf, sr.F32, False)):
        src = torch.from_numpy(arr)
        if pin:
            src = src.pin_memory()
        out = np.zeros(1, np.int64 if dt == sr.I32 else np.float32)
        sr.check(sr.reduce_sum_host_ptr(src.data_ptr() if n else arr.ctypes.data, n, dt, out.ctypes.data, None))
        if dt == sr.I32:
            assert int(out[0]) == oracle.sum_i32(arr)
        else:
            ex = oracle.to_float(oracle.exact_f32(arr))
            assert abs(float(out[0]) - ex) <= oracle.stated_fp32_bound(oracle.sum_abs_f32(arr))


def test_host_entry_flags_and_repeat(sr):
    x = workloads.cancelling_f32(1 << 24, cond=1e6, seed=1)
    pinned = torch.from_numpy(x).pin_memory()
    S = oracle.to_float(oracle.exact_f32(x))
    out = np.zeros(1, np.float64)
    cfg = sr.make_config(sr.F_KAHAN | sr.F_FP64_COMBINE)
    vals = set()
    for _ in range(3):
        sr.check(sr.reduce_sum_host_ptr(pinned.data_ptr(), x.size, sr.F32, out.ctypes.data, cfg))
        vals.add(float(out[0]))
        assert abs(float(out[0]) - S) / abs(S) <= 1e-6
    assert len(vals) == 1


def test_host_direct_reads(sr):
    """SR_F_HOST_DIRECT: the kernel reads page-locked host memory in place."""
    n = (1 << 24) + 3
    x = workloads.uniform_f32(n, seed=9)
    xi = workloads.uniform_i32(n, seed=9)
    pinned = torch.from_numpy(x).pin_memory()
    pinned_i = torch.from_numpy(xi).pin_memory()
    out = np.zeros(1, np.float32)
    outi = np.zeros(1, np.int64)
    cfg = sr.make_config(sr.F_HOST_DIRECT)
    sr.check(sr.reduce_sum_host_ptr(pinned.data_ptr(), n, sr.F32, out.ctypes.data, cfg))
    ex = oracle.to_float(oracle.exact_f32(x))
    assert abs(float(out[0]) - ex) <= oracle.stated_fp32_bound(oracle.sum_abs_f32(x))
    sr.check(sr.reduce_sum_host_ptr(pinned_i.data_ptr() + 4, n - 1, sr.I32, outi.ctypes.data, cfg))
    assert int(outi[0]) == oracle.sum_i32(xi[1:])
    # device memory is not a host array
    d = torch.from_numpy(x).cuda()
    assert sr.reduce_sum_host_ptr(d.data_ptr(), n, sr.F32, out.ctypes.data, cfg) == sr.ERR_ARG
