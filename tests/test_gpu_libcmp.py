"""The CUB comparison library used by the benchmark suites computes the
same sums as the library (int32 bit-exact; FP32 within the stated bound), so
the sweep compares like with like."""
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_cub_reference_matches(sr):
    import libcmp
    libcmp.build()
    cmp = libcmp.lib()
    libcmp.check(cmp.cmp_prepare(1 << 22), "cmp_prepare")
    st = torch.cuda.current_stream().cuda_stream
    for n in (1, 1000, (1 << 22) - 3):
        xi = workloads.uniform_i32(n, seed=n)
        x = workloads.uniform_f32(n, seed=n)
        xid, xd = torch.from_numpy(xi).cuda(), torch.from_numpy(x).cuda()
        oi = torch.zeros((), dtype=torch.int64, device="cuda")
        of = torch.zeros((), dtype=torch.float32, device="cuda")
        libcmp.check(cmp.cmp_cub_sum_i32(xid.data_ptr(), n, oi.data_ptr(), st), "cub i32")
        libcmp.check(cmp.cmp_cub_sum_f32(xd.data_ptr(), n, of.data_ptr(), st), "cub f32")
        assert int(oi.item()) == oracle.sum_i32(xi) == int(sr.reduce_sum(xid).item())
        exact = oracle.to_float(oracle.exact_f32(x))
        assert abs(float(of.item()) - exact) <= oracle.stated_fp32_bound(oracle.sum_abs_f32(x))
