"""sr_reduce_sum_noalloc: the sum for callers that cannot allocate device
memory (no cudaMalloc available or allowed where they run).  It keeps its
scratch in one fixed device array inside the library instead of a workspace
allocated on first use.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import workloads

ALIGNED = 1 << 20   # stand-in device address: never dereferenced on the host


def test_noalloc_rejects_without_touching_the_gpu(sr):
    def call(**kw):
        return sr.reduce_sum_noalloc_ptr(ALIGNED, 1000, sr.F32, ALIGNED, sr.make_config(**kw), stream=0)
    assert call(variant=sr.TWO_KERNEL) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.ATOMIC) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.LAST_BLOCK | sr.F_BULK) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.LAST_BLOCK, grid=4097) == sr.ERR_ARG          # above the 4096-unit maximum
    assert call(variant=sr.LAST_BLOCK | sr.CLUSTER(1), grid=8194) == sr.ERR_ARG
    assert sr.reduce_sum_noalloc_ptr(ALIGNED, -1, sr.F32, ALIGNED, None, stream=0) == sr.ERR_ARG
    # the TMA ring waits on mbarriers and could report a timeout, which this
    # entry point has no error word for: refused in every spelling
    assert call(variant=sr.AUTO | sr.F_BULK) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.LAST_BLOCK | sr.F_BULK | sr.F_KAHAN) == sr.ERR_UNSUPPORTED


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point(sr):
    """Two calls in a row through the C ABI agree with sr_reduce_sum_ex's
    last-block-done result: within the FP32 gate the parity tests use for
    binary32 input, exactly for int32 input."""
    import torch
    cases = [(workloads.uniform_f32((1 << 20) + 3, seed=21), sr.F32),
             (workloads.uniform_f32(1 << 24, seed=22), sr.F32),
             (workloads.uniform_i32((1 << 22) + 1, seed=23), sr.I32)]
    for x_np, dt in cases:
        x = torch.from_numpy(x_np).cuda()
        odt = torch.int64 if dt == sr.I32 else torch.float32
        ref = torch.empty((), dtype=odt, device="cuda")
        sr.check(sr.reduce_sum_ptr(x.data_ptr(), x.numel(), dt, ref.data_ptr(), sr.make_config(sr.LAST_BLOCK)))
        for _ in range(2):
            out = torch.full((), -7, dtype=odt, device="cuda")
            sr.check(sr.reduce_sum_noalloc_ptr(x.data_ptr(), x.numel(), dt, out.data_ptr(), None))
            torch.cuda.synchronize()
            if dt == sr.I32:
                assert int(out.item()) == int(ref.item()) == oracle.sum_i32(x_np)
            else:
                bound = oracle.stated_fp32_bound(oracle.sum_abs_f32(x_np))
                assert abs(float(out.item()) - float(ref.item())) <= bound
                assert abs(float(out.item()) - oracle.to_float(oracle.exact_f32(x_np))) <= bound


@pytest.mark.gpu
def test_noalloc_flags_clusters_and_largest_grid(sr):
    """The options the header says are honoured, each on two calls in a row
    against sr_reduce_sum_ex with the same configuration: a cluster size, the
    compensated path, the binary64 combine (8-byte output), and an explicit
    grid of exactly the 4096-unit maximum; binary32 results within the
    stated gate of the exact sum, int32 exactly."""
    import torch
    n = (1 << 22) + 5
    xf = workloads.uniform_f32(n, seed=31)
    xi = workloads.uniform_i32(n, seed=32)
    exact = oracle.to_float(oracle.exact_f32(xf))
    bound = oracle.stated_fp32_bound(oracle.sum_abs_f32(xf))
    dfx, dix = torch.from_numpy(xf).cuda(), torch.from_numpy(xi).cuda()
    cases = [(sr.LAST_BLOCK | sr.CLUSTER(1), {}, torch.float32),
             (sr.LAST_BLOCK | sr.CLUSTER(3), {}, torch.float32),
             (sr.LAST_BLOCK | sr.F_KAHAN, {}, torch.float32),
             (sr.LAST_BLOCK | sr.F_KAHAN | sr.F_FP64_COMBINE, {}, torch.float64),
             (sr.LAST_BLOCK | sr.F_FP64_COMBINE, {}, torch.float64),
             (sr.LAST_BLOCK, {"grid": 4096, "block_threads": 256}, torch.float32),
             (sr.LAST_BLOCK | sr.CLUSTER(1), {"grid": 8192, "block_threads": 128}, torch.float32)]
    for variant, kw, odt in cases:
        cfg = sr.make_config(variant, **kw)
        ref = torch.empty((), dtype=odt, device="cuda")
        sr.check(sr.reduce_sum_ptr(dfx.data_ptr(), n, sr.F32, ref.data_ptr(), cfg))
        for _ in range(2):
            out = torch.full((), -7, dtype=odt, device="cuda")
            sr.check(sr.reduce_sum_noalloc_ptr(dfx.data_ptr(), n, sr.F32, out.data_ptr(), cfg))
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - exact) <= bound, (hex(variant), kw, got, exact)
            assert abs(got - float(ref.item())) <= bound, (hex(variant), kw)
        refi = torch.empty((), dtype=torch.int64, device="cuda")
        sr.check(sr.reduce_sum_ptr(dix.data_ptr(), n, sr.I32, refi.data_ptr(), cfg))
        outi = torch.full((), -7, dtype=torch.int64, device="cuda")
        sr.check(sr.reduce_sum_noalloc_ptr(dix.data_ptr(), n, sr.I32, outi.data_ptr(), cfg))
        torch.cuda.synchronize()
        assert int(outi.item()) == int(refi.item()) == oracle.sum_i32(xi), (hex(variant), kw)
