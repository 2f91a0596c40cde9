"""Failure detection without a GPU fault: a device wait on a flag nothing sets
expires by its own bound, the host reads SR_ERR_TIMEOUT, and the context
keeps working."""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(sr):
    s = torch.cuda.Stream()
    assert sr.stream_status(s) == sr.OK
    t0 = time.perf_counter()
    assert sr.selftest_bounded_wait(20_000_000, s) == sr.OK      # 20 ms bound
    assert sr.stream_status(s) == sr.ERR_TIMEOUT                 # synchronises, reads, clears
    assert time.perf_counter() - t0 < 5.0
    assert sr.stream_status(s) == sr.OK                          # cleared
    # the context is intact: a full reduction on the same stream still matches the oracle
    x = workloads.uniform_i32(1 << 22, seed=5)
    xd = torch.from_numpy(x).cuda()
    with torch.cuda.stream(s):
        out = sr.reduce_sum(xd, variant=sr.LAST_BLOCK | sr.F_BULK, stream=s)
    s.synchronize()
    assert int(out.item()) == oracle.sum_i32(x)
    # and so is the segmented path with per-segment tickets (reset with the error)
    off = workloads.segment_offsets(40_000, 1 << 22, seed=5, median=100, sigma=1.5, lo=0, hi=1 << 16)
    xs = workloads.uniform_i32(int(off[-1]), seed=5)
    xsd, od = torch.from_numpy(xs).cuda(), torch.from_numpy(off).cuda()
    with torch.cuda.stream(s):
        got = sr.reduce_sum_segmented(xsd, od, variant=sr.LAST_BLOCK, stream=s)   # the TMA form
    s.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.segsum_i32(xs, off))
    assert sr.stream_status(s) == sr.OK


def test_selftest_rejects_bad_limits(sr):
    assert sr.selftest_bounded_wait(0) == sr.ERR_ARG
    assert sr.selftest_bounded_wait(20_000_000_000) == sr.ERR_ARG


def test_stream_release_and_reuse(sr):
    """Workspaces and staging buffers of a stream are freed on request and
    re-created by the next call on it."""
    x = workloads.uniform_i32(1 << 20, seed=6)
    xd = torch.from_numpy(x).cuda()
    pinned = torch.from_numpy(x).pin_memory()
    host_out = np.zeros(1, np.int64)
    for _ in range(3):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            out = sr.reduce_sum(xd, variant=sr.LAST_BLOCK, stream=s)
        sr.check(sr.reduce_sum_host_ptr(pinned.data_ptr(), x.size, sr.I32, host_out.ctypes.data, None, s))
        s.synchronize()
        assert int(out.item()) == int(host_out[0]) == oracle.sum_i32(x)
        assert sr.stream_release(s) == sr.OK
        with torch.cuda.stream(s):
            out = sr.reduce_sum(xd, variant=sr.LAST_BLOCK, stream=s)   # workspace re-created
        s.synchronize()
        assert int(out.item()) == oracle.sum_i32(x)
        assert sr.stream_release(s) == sr.OK
