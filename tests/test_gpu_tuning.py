"""The autotuner, the planner's SR_AUTO regimes and the performance-model
selector on the device."""
import math

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def test_plan_auto_regimes(sr):
    """SR_AUTO: one CTA up to 32 KiB and a cluster of up to 16 CTAs up to
    1 MiB (one 16 B x 2 batch per thread), the two-kernel form up to 512 MiB,
    then last-block-done on the TMA ring (FP32 sizes; the ring's shape per
    dtype)."""
    cases = [(1 << 10, sr.SINGLE_CLUSTER, 0), (1 << 12, sr.SINGLE_CLUSTER, 0), (1 << 14, sr.SINGLE_CLUSTER, 3),
             (1 << 18, sr.SINGLE_CLUSTER, 4), (1 << 20, sr.TWO_KERNEL, 0), (1 << 24, sr.TWO_KERNEL, 0),
             (1 << 26, sr.TWO_KERNEL, 0), (1 << 27, sr.TWO_KERNEL, 0), (1 << 28, sr.LAST_BLOCK, 0)]
    for n, stage, log2c in cases:
        r = sr.plan(n, sr.F32)
        assert r.variant & sr.STAGE_MASK == stage, n
        assert (r.variant & sr.CLUSTER_MASK) >> sr.CLUSTER_SHIFT == log2c, n
    r = sr.plan(1 << 27, sr.F32)
    assert (r.vec_bytes, r.unroll, r.block_threads) == (16, 1, 512) and not r.variant & sr.F_BULK
    # plain, 1-64 MiB: 256-bit loads; below 4 MiB 16 KiB per CTA (BF16 / FP8: 512 x 16 B x 2)
    for n, dt, shape in (((1 << 19), sr.F32, (32, 2, 256)), ((1 << 20), sr.BF16, (16, 2, 512)),
                         ((1 << 21), sr.FP8E4M3, (16, 2, 512)),
                         ((1 << 20), sr.F32, (32, 2, 512))):
        r = sr.plan(n, dt)
        assert (r.vec_bytes, r.unroll, r.block_threads) == shape, (n, dt, r.as_dict())
    # int32, 1-64 MiB: exact in any order, so the atomic finish from 4 MiB (256 x 32 B x 4, x 8 from 32 MiB)
    for n, stage, shape in (((1 << 19), sr.TWO_KERNEL, (16, 4, 256)), ((1 << 20), sr.ATOMIC, (32, 4, 256)),
                            ((1 << 22), sr.ATOMIC, (32, 4, 256)), ((1 << 24), sr.ATOMIC, (32, 8, 256))):
        r = sr.plan(n, sr.I32)
        assert r.variant & sr.STAGE_MASK == stage and (r.vec_bytes, r.unroll, r.block_threads) == shape, \
            (n, r.as_dict())
    for n, shape in (((1 << 10), (1, 128, 2)), ((1 << 12), (1, 512, 2)), ((1 << 14), (8, 256, 2)),
                     ((1 << 16), (16, 512, 2)), ((1 << 18), (16, 1024, 4))):
        r = sr.plan(n, sr.F32)
        assert (r.grid, r.block_threads, r.unroll, r.vec_bytes) == shape + (16,), (n, r.as_dict())
    r = sr.plan(1 << 28, sr.F32)
    assert r.variant & sr.F_BULK and (r.tile_bytes, r.stages, r.block_threads) == (65536, 2, 288)
    r = sr.plan(1 << 28, sr.I32)
    assert r.variant & sr.F_BULK and (r.tile_bytes, r.stages, r.block_threads) == (32768, 4, 160)
    r = sr.plan(1 << 30, sr.FP8E4M3)
    assert r.variant & sr.F_BULK and (r.tile_bytes, r.stages, r.block_threads) == (65536, 3, 288)
    r = sr.plan(1 << 28, sr.FP8E4M3)
    assert (r.vec_bytes, r.unroll, r.block_threads) == (16, 4, 512) and not r.variant & sr.F_BULK
    r = sr.plan(1 << 28, sr.F32, sr.make_config(sr.F_KAHAN))
    assert r.variant & sr.F_BULK and r.tile_bytes == 32768 and r.stages == 4
    # compensated, 1-64 MiB: 256-bit loads; 256 x 2 below 8 MiB, 1024 x 4 to 32 MiB, 1024 x 8 (FP8 x 4) above
    for n, dt, shape in (((1 << 19), sr.F32, (32, 2, 256)), ((1 << 22), sr.F32, (32, 4, 1024)),
                         ((1 << 24), sr.F32, (32, 8, 1024)), ((1 << 21), sr.BF16, (32, 2, 256)),
                         ((1 << 25), sr.BF16, (32, 8, 1024)), ((1 << 26), sr.FP8E4M3, (32, 4, 1024))):
        r = sr.plan(n, dt, sr.make_config(sr.F_KAHAN))
        assert (r.vec_bytes, r.unroll, r.block_threads) == shape, (n, dt, r.as_dict())
    # explicit fields override the table; a vector width or unroll selects the LDG path
    r = sr.plan(1 << 28, sr.F32, sr.make_config(sr.AUTO, vec_bytes=32, unroll=2))
    assert (r.vec_bytes, r.unroll) == (32, 2) and not r.variant & sr.F_BULK


def test_autotune_times_every_candidate(sr):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 1 << 24
    x = torch.from_numpy(workloads.uniform_f32(n, seed=1)).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cands = sr.candidates(sms)
    us = sr.autotune(x.data_ptr(), n, sr.F32, out.data_ptr(), cands, reps=2)
    assert len(us) == len(cands)
    finite = [u for u in us if math.isfinite(u)]
    assert len(finite) >= 30 and all(0 < u < 10_000 for u in finite)
    # candidates that cannot run are marked, not fatal: a grid.sync grid larger
    # than what can be co-resident
    bad = (sr.Config * 1)(sr.make_config(sr.GRID_SYNC, grid=sms * 64, block_threads=1024))
    assert math.isinf(sr.autotune(x.data_ptr(), n, sr.F32, out.data_ptr(), bad, reps=1)[0])
    # segmented form
    off = workloads.segment_offsets(1000, n, seed=2, median=4096, sigma=1.5, hi=1 << 22)
    od = torch.from_numpy(off).cuda()
    outs = torch.zeros(1000, dtype=torch.float64, device="cuda")
    us = sr.autotune(x.data_ptr(), int(off[-1]), sr.F32, outs.data_ptr(), cands, reps=2,
                     offsets_ptr=od.data_ptr(), nseg=1000)
    assert sum(math.isfinite(u) for u in us) >= 30


def test_model_selector_picks_a_reasonable_candidate(sr):
    """The performance model's choice is within 2x of the best measured
    candidate at a large and a small size (it is the baseline, not the goal)."""
    from paper_2004_05371_gb300 import selector
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cands = sr.candidates(sms)
    params = selector.default_model_params(sms)
    for n in (1 << 26, 1 << 14):
        x = torch.from_numpy(workloads.uniform_f32(n, seed=3)).cuda()
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        us = np.array(sr.autotune(x.data_ptr(), n, sr.F32, out.data_ptr(), cands, reps=3))
        i, pred = sr.select_analytic(params, n, sr.F32, 1, cands)
        assert np.isfinite(us[i]) and us[i] <= 2.0 * np.min(us), (n, us[i], np.min(us))


def test_model_selector_never_picks_a_rejected_launch(sr):
    """A grid.sync() candidate whose grid cannot be co-resident is rejected by
    the planner (Section VIII-B), so the model never chooses it — even when
    its formula alone would rank it first — and predicts +inf for it; the
    same holds for the segmented planner."""
    from paper_2004_05371_gb300 import selector
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    params = selector.default_model_params(sms)
    params.grid_sync_ns = 0.0                   # makes grid.sync the model's favourite
    too_big = sr.make_config(sr.GRID_SYNC, grid=64 * sms, block_threads=1024, vec_bytes=32, unroll=8)
    fits = sr.make_config(sr.LAST_BLOCK, grid=sms, block_threads=256, vec_bytes=16, unroll=1)
    cands = (sr.Config * 2)(too_big, fits)
    for nseg in (1, 1000):
        i, pred = sr.select_analytic(params, 1 << 26, sr.F32, nseg, cands)
        assert i == 1 and math.isinf(pred[0]) and math.isfinite(pred[1]), nseg
    with pytest.raises(sr.SRError):
        sr.select_analytic(params, 1 << 26, sr.F32, 1, (sr.Config * 1)(too_big))
    # every choice over the standard candidate set is a launch the planner accepts
    cands = sr.candidates(sms)
    for n in (1 << 12, 1 << 20, 1 << 28):
        for nseg in (1, 10, 10_000):
            i, _ = sr.select_analytic(params, n, sr.F32, nseg, cands)
            if nseg > 1:
                sr.plan_segmented(nseg, sr.F32, cands[i])
            else:
                sr.plan(n, sr.F32, cands[i])
