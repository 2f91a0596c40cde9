"""Parity of the segmented (batched) sum with the CPU oracle, segment by segment.

int32: bit-exact per segment.  binary32 (random-sign data): per segment
|err| <= 4 eps32 sum|x_seg| (the stated plain-tree gate), and within the
compensated bound with SR_F_KAHAN.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

STAGES = [1, 2, 3, 4]  # two-kernel, atomic, last-block, grid-sync
DENSE = 0x2000  # SR_F_DENSE_SEGMENTS: the warp-wide segmented scan over rows with many boundaries
EPS32 = 2.0 ** -23
U = 2.0 ** -24


def _dev(a, offset=0):
    buf = torch.zeros(a.size + offset + 8, dtype=torch.from_numpy(a[:0]).dtype, device="cuda")
    v = buf[offset:offset + a.size]
    if a.size:
        v.copy_(torch.from_numpy(a))
    return v


def _check(sr, x, off, variant, x_off=0, **cfg):
    """Run one segmented call and compare every segment with the oracle."""
    if x.size == 0:  # x must be a valid pointer whenever nseg > 0 (empty torch views have none)
        x = np.zeros(1, x.dtype)
    xd = _dev(x, x_off)
    od = torch.from_numpy(off).cuda()
    out = sr.reduce_sum_segmented(xd, od, config=sr.make_config(variant, **cfg))
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    if x.dtype == np.int32:
        ref = oracle.segsum_i32(x, off)
        bad = np.nonzero(got != ref)[0]
        assert bad.size == 0, (variant, cfg, bad[:5], got[bad[:5]], ref[bad[:5]])
    else:
        ex = oracle.segexact_f32(x, off)
        sabs = oracle.segsum_abs_f32(x, off)
        tol = (2 * U + np.diff(off) * U * U) * sabs if variant & sr.F_KAHAN else 4 * EPS32 * sabs
        err = np.abs(got.astype(np.float64) - ex)
        bad = np.nonzero(err > tol)[0]
        assert bad.size == 0, (variant, cfg, bad[:5], got[bad[:5]], ex[bad[:5]])
    return got


@pytest.mark.parametrize("stage", STAGES)
@pytest.mark.parametrize("nseg,max_len", [(1, 0), (1, 1), (1, 100_000), (2, 5), (31, 0), (33, 7),
                                          (500, 300), (5000, 40), (300, 20_000)])
def test_random_layouts(sr, stage, nseg, max_len):
    off = workloads.random_segment_offsets(nseg, max_len, seed=nseg + max_len)
    n = int(off[-1])
    xf = workloads.uniform_f32(n, seed=1)
    xi = workloads.uniform_i32(n, seed=1)
    for grid in (0, 1, 3):
        for x_off in (0, 1):
            for dense in (0, DENSE):
                _check(sr, xi, off, stage | dense, x_off, grid=grid)
                _check(sr, xf, off, stage | dense, x_off, grid=grid)


@pytest.mark.parametrize("stage", STAGES)
@pytest.mark.parametrize("vec,unroll,block", [(16, 1, 32), (16, 4, 256), (32, 2, 512), (32, 8, 512), (16, 8, 128),
                                              (32, 8, 256)])
def test_launch_shapes(sr, stage, vec, unroll, block):
    off = workloads.segment_offsets(300, 1 << 20, seed=5, median=1024, sigma=2.0, hi=1 << 18)
    n = int(off[-1])
    _check(sr, workloads.uniform_i32(n, seed=2), off, stage, vec_bytes=vec, unroll=unroll, block_threads=block)
    _check(sr, workloads.uniform_f32(n, seed=2), off, stage, 3, vec_bytes=vec, unroll=unroll, block_threads=block)


def test_base_offset_and_trailing_empty_segments(sr):
    off = np.array([5, 5, 9, 9, 100, 1000, 1000, 1000], dtype=np.int64)
    x = workloads.uniform_i32(1000, seed=3)
    for st in STAGES:
        for grid in (0, 1, 2, 64):
            _check(sr, x, off, st, grid=grid)


def test_all_empty_and_single_element_segments(sr):
    off = np.zeros(1001, np.int64)
    x = np.zeros(0, np.int32)
    for st in STAGES:
        got = _check(sr, np.zeros(1, np.int32), off, st)
        assert not got.any()
    off = np.arange(100_001, dtype=np.int64)
    x = workloads.uniform_i32(100_000, seed=4)
    for st in STAGES:
        got = _check(sr, x, off, st)
        assert np.array_equal(got, x.astype(np.int64))


def test_one_segment_spans_every_warp(sr):
    n = (1 << 22) + 3
    off = np.array([0, n], np.int64)
    x = workloads.uniform_f32(n, seed=6)
    xi = workloads.uniform_i32(n, seed=6)
    for st in STAGES:
        _check(sr, xi, off, st)
        _check(sr, x, off, st)
    off3 = np.array([0, 1, n - 1, n], np.int64)
    for st in STAGES:
        _check(sr, xi, off3, st)


@pytest.mark.parametrize("flags", [0x100, 0x300, 0x200])
def test_precision_flags(sr, flags):
    off = workloads.segment_offsets(2000, 1 << 21, seed=8, median=512, sigma=2.0, hi=1 << 19)
    x = workloads.lognormal_f32(int(off[-1]), seed=8, sigma=3.0)
    for st in STAGES:
        _check(sr, x, off, st | flags)


def test_bf16_and_fp8_segments(sr):
    off = workloads.random_segment_offsets(700, 3000, seed=9)
    n = int(off[-1])
    x = workloads.lognormal_f32(n, seed=9, sigma=2.0)
    bits = workloads.to_bf16_bits(x)
    codes, deq = workloads.to_e4m3_codes(x)
    od = torch.from_numpy(off).cuda()
    dec_b = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
    xd_b = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    xd_f = torch.from_numpy(codes).cuda()
    dec_f = (torch.from_numpy(codes).view(torch.float8_e4m3fn).float() * deq).numpy()
    for st in STAGES:
        got = sr.reduce_sum_segmented(xd_b, od, variant=st).cpu().numpy()
        ex = oracle.segexact_f32(dec_b, off)
        assert np.all(np.abs(got - ex) <= 4 * EPS32 * oracle.segsum_abs_f32(dec_b, off) + 1e-30)
        got = sr.reduce_sum_segmented(xd_f, od, config=sr.make_config(st, scale=deq)).cpu().numpy()
        for s in range(700):  # every segment against its exact sum
            a, b = off[s], off[s + 1]
            exs = oracle.to_float(oracle.exact_e4m3(codes[a:b], deq))
            sabs = float(np.abs(dec_f[a:b]).astype(np.float64).sum())
            assert abs(got[s] - exs) <= 4 * EPS32 * sabs * 1.001 + 1e-30


def test_deterministic_and_graph_replay(sr):
    off = workloads.segment_offsets(3000, 1 << 22, seed=10, median=512, sigma=2.0, hi=1 << 20)
    n = int(off[-1])
    x = workloads.uniform_f32(n, seed=10)
    xd, od = _dev(x), torch.from_numpy(off).cuda()
    for st in (1, 3, 4):
        outs = [sr.reduce_sum_segmented(xd, od, variant=st).cpu().numpy() for _ in range(3)]
        assert all(np.array_equal(outs[0], o) for o in outs[1:])
    ref = sr.reduce_sum_segmented(xd, od, variant=sr.LAST_BLOCK).cpu().numpy()
    out = torch.full((off.size - 1,), -1.0, dtype=torch.float32, device="cuda")
    g = sr.SegmentedGraph(xd, od, out, sr.make_config(sr.LAST_BLOCK))
    for _ in range(3):
        out.fill_(-1.0)
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
    g.close()
    assert sr.stream_status() == sr.OK


@pytest.mark.slow
def test_full_size_lognormal_10k_segments(sr):
    """10,000 segments, lengths lognormal (median 4096, sigma 1.94, clipped to
    [1, 2^24]), about 2^28 elements: every segment against the oracle."""
    off = workloads.segment_offsets(10_000, 1 << 28, seed=0)
    n = int(off[-1])
    x = workloads.uniform_f32(n, seed=0)
    xd, od = _dev(x), torch.from_numpy(off).cuda()
    ex = oracle.segexact_f32(x, off)
    tol = 4 * EPS32 * oracle.segsum_abs_f32(x, off)
    for st in STAGES:
        got = sr.reduce_sum_segmented(xd, od, variant=st).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ex) <= tol), st


@pytest.mark.parametrize("nseg", [32, 64, 1024, 1056, 32 * 33])
def test_search_with_exactly_32_candidates_left(sr, nseg):
    """Layouts where a warp's segment search ends with exactly 32 candidates
    that all start before its piece: nseg - 1 one-element segments, then one
    long segment covering every later warp."""
    n_long = 1 << 20
    lens = np.ones(nseg, np.int64)
    lens[-1] = n_long
    off = np.zeros(nseg + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    x = workloads.uniform_i32(int(off[-1]), seed=nseg)
    xf = workloads.uniform_f32(int(off[-1]), seed=nseg)
    for st in STAGES:
        for grid in (0, 4, 64):
            _check(sr, x, off, st, grid=grid)
            _check(sr, xf, off, st, grid=grid)
    rng = np.random.default_rng(nseg)
    off2 = np.zeros(nseg + 1, np.int64)
    np.cumsum(rng.integers(0, 3, nseg) * (rng.random(nseg) < 0.97) + (rng.random(nseg) < 0.03) * 50_000,
              out=off2[1:])
    x2 = workloads.uniform_i32(int(off2[-1]) + 1, seed=1)
    for st in STAGES:
        _check(sr, x2, off2, st)


@pytest.mark.parametrize("stage", STAGES)
@pytest.mark.parametrize("seg_len", [3, 5, 8, 9, 16, 31, 100, 255, 257])
def test_rows_with_many_boundaries(sr, stage, seg_len):
    """Rows in which many segments end: at most one boundary per lane takes
    the warp-wide segmented scan, two or more in a lane the per-segment path
    (lengths below the lane vector); both launch-shape families, aligned and
    misaligned data; bit-exact for int32, within the gates for binary32."""
    nseg = (1 << 18) // seg_len
    off = np.arange(nseg + 1, dtype=np.int64) * seg_len
    n = int(off[-1])
    xi = workloads.uniform_i32(n, seed=seg_len)
    xf = workloads.uniform_f32(n, seed=seg_len)
    for dense in (0, DENSE):
        for vec, unroll, block in ((32, 8, 256), (16, 2, 128)):
            for x_off in (0, 1):
                _check(sr, xi, off, stage | dense, x_off, vec_bytes=vec, unroll=unroll, block_threads=block)
                _check(sr, xf, off, stage | dense, x_off, vec_bytes=vec, unroll=unroll, block_threads=block)
        _check(sr, xf, off, stage | 0x100 | dense)
        _check(sr, xf, off, stage | 0x300 | dense)


@pytest.mark.parametrize("stage", STAGES)
def test_many_small_lognormal_segments(sr, stage):
    """100,000 lognormal segments (median 40 elements, empty ones included)
    over ~2^22 elements: rows mixing both boundary paths, every dtype."""
    off = workloads.segment_offsets(100_000, 1 << 22, seed=12, median=40, sigma=1.5, lo=0, hi=1 << 16)
    n = int(off[-1])
    x = workloads.lognormal_f32(n, seed=12, sigma=2.0)
    bits = workloads.to_bf16_bits(x)
    dec_b = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
    codes, deq = workloads.to_e4m3_codes(x)
    od = torch.from_numpy(off).cuda()
    xd_b = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    xd_f = torch.from_numpy(codes).cuda()
    ex_b = oracle.segexact_f32(dec_b, off)
    gate_b = 4 * EPS32 * oracle.segsum_abs_f32(dec_b, off) + 1e-30
    for dense in (0, DENSE):
        _check(sr, workloads.uniform_i32(n, seed=12), off, stage | dense)
        _check(sr, workloads.uniform_f32(n, seed=12), off, stage | dense)
        got = sr.reduce_sum_segmented(xd_b, od, variant=stage | dense).cpu().numpy()
        assert np.all(np.abs(got - ex_b) <= gate_b), dense
        got = sr.reduce_sum_segmented(xd_f, od, config=sr.make_config(stage | dense, scale=deq)).cpu().numpy()
        for s in range(0, 100_000, 997):
            a, b = off[s], off[s + 1]
            exs = oracle.to_float(oracle.exact_e4m3(codes[a:b], deq))
            sabs = oracle.sum_e4m3(codes[a:b] & 0x7F, deq)
            assert abs(got[s] - exs) <= 4 * EPS32 * sabs * 1.001 + 1e-30, (dense, s)


BULK = 0x400  # SR_F_BULK: each warp streams its piece through a TMA ring in shared memory


@pytest.mark.parametrize("stage", STAGES)
@pytest.mark.parametrize("vec,unroll,stages,block", [(32, 4, 3, 256), (32, 2, 2, 64), (32, 8, 2, 256),
                                                     (16, 4, 4, 128), (16, 8, 3, 256), (32, 4, 8, 32)])
def test_bulk_ring(sr, stage, vec, unroll, stages, block):
    """The TMA form of the segmented kernel: random layouts with empty, tiny and
    long segments, aligned and misaligned data, every grid stage and ring
    shape; bit-exact for int32, within the gates for binary32 (plain and
    compensated)."""
    for nseg, max_len in ((1, 100_000), (33, 7), (5000, 40), (300, 20_000)):
        off = workloads.random_segment_offsets(nseg, max_len, seed=nseg + max_len + unroll)
        n = int(off[-1])
        xi = workloads.uniform_i32(n, seed=7)
        xf = workloads.uniform_f32(n, seed=7)
        for x_off in (0, 1):
            cfg = dict(vec_bytes=vec, unroll=unroll, stages=stages, block_threads=block)
            _check(sr, xi, off, stage | BULK, x_off, **cfg)
            _check(sr, xf, off, stage | BULK, x_off, **cfg)
        _check(sr, xf, off, stage | BULK | 0x100, **cfg)


def test_bulk_ring_dtypes_and_plan(sr):
    off = workloads.segment_offsets(2000, 1 << 21, seed=13, median=512, sigma=2.0, hi=1 << 19)
    n = int(off[-1])
    x = workloads.lognormal_f32(n, seed=13, sigma=2.0)
    bits = workloads.to_bf16_bits(x)
    dec_b = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
    codes, deq = workloads.to_e4m3_codes(x)
    od = torch.from_numpy(off).cuda()
    xd_b = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    xd_f = torch.from_numpy(codes).cuda()
    for st in STAGES:
        got = sr.reduce_sum_segmented(xd_b, od, variant=st | BULK).cpu().numpy()
        assert np.all(np.abs(got - oracle.segexact_f32(dec_b, off)) <=
                      4 * EPS32 * oracle.segsum_abs_f32(dec_b, off) + 1e-30)
        got = sr.reduce_sum_segmented(xd_f, od, config=sr.make_config(st | BULK, scale=deq)).cpu().numpy()
        for s in range(0, 2000, 97):
            a, b = off[s], off[s + 1]
            exs = oracle.to_float(oracle.exact_e4m3(codes[a:b], deq))
            assert abs(got[s] - exs) <= 4 * EPS32 * oracle.sum_e4m3(codes[a:b] & 0x7F, deq) * 1.001 + 1e-30
    r = sr.plan_segmented(2000, sr.F32, sr.make_config(sr.LAST_BLOCK | BULK))
    assert r.variant & BULK and r.unroll == 4 and r.stages == 2
    with pytest.raises(sr.SRError):   # the TMA form has no dense pass
        sr.plan_segmented(2000, sr.F32, sr.make_config(sr.LAST_BLOCK | BULK | DENSE))
    with pytest.raises(sr.SRError) as e:  # 16 warps x 2 stages x 8 KiB: more shared memory than a CTA has
        sr.plan_segmented(2000, sr.F32, sr.make_config(sr.LAST_BLOCK | BULK, block_threads=512, unroll=8, stages=2))
    assert e.value.status == sr.ERR_LAUNCH


def test_default_load_path_by_segment_count(sr):
    """Without an explicit shape, 32768 or more segments take the TMA form,
    fewer the LDG one; any explicit shape field keeps the LDG path."""
    assert sr.plan_segmented(32767, sr.F32).variant & BULK == 0
    r = sr.plan_segmented(32768, sr.F32)
    assert r.variant & BULK and (r.unroll, r.stages) == (4, 2)
    assert sr.plan_segmented(100_000, sr.F32, sr.make_config(sr.ATOMIC, unroll=8)).variant & BULK == 0
    off = workloads.segment_offsets(40_000, 1 << 22, seed=14, median=100, sigma=1.5, lo=0, hi=1 << 16)
    n = int(off[-1])
    for st in STAGES:
        _check(sr, workloads.uniform_i32(n, seed=14), off, st)
        _check(sr, workloads.uniform_f32(n, seed=14), off, st, 1)


WARP = 0x4000  # SR_F_WARPSEGMENTS: whole segments per warp, no grid stage


LANE = 0x8000  # SR_F_LANE_SEGMENTS: whole segments per thread, no grid stage
ADAPT = 0x10000  # SR_F_ADAPTIVE_SEGMENTS: lanes / warps / queued chunks, one cooperative launch


@pytest.mark.parametrize("form,vec,unroll,block", [
    (WARP, 16, 4, 256), (WARP, 32, 1, 64), (WARP, 16, 8, 512), (WARP, 32, 2, 128), (WARP, 16, 1, 32),
    (WARP, 32, 8, 256), (LANE, 16, 4, 256), (LANE, 16, 1, 32), (LANE, 32, 8, 512), (LANE, 16, 2, 128),
    (LANE, 32, 4, 256), (LANE, 32, 1, 64)])
def test_warp_segments(sr, form, vec, unroll, block):
    """The whole-segment forms (a warp, or a single thread, per segment):
    random layouts with empty, tiny and long segments (one of 100,000
    elements summed by a single warp or thread), aligned and misaligned data,
    grids from one CTA (32 segments per warp block) to the default; the stage
    bits change nothing.  Bit-exact for int32, within the gates for binary32
    (plain, compensated, binary64 output)."""
    for nseg, max_len in ((1, 100_000), (2, 5), (33, 7), (500, 300), (5000, 40), (300, 20_000)):
        off = workloads.random_segment_offsets(nseg, max_len, seed=nseg + max_len + vec)
        n = int(off[-1])
        xi = workloads.uniform_i32(n, seed=17)
        xf = workloads.uniform_f32(n, seed=17)
        shape = dict(vec_bytes=vec, unroll=unroll, block_threads=block)
        for grid in (0, 1, 3):
            for x_off in (0, 1, 3):
                _check(sr, xi, off, form | STAGES[(grid + x_off) % 4], x_off, grid=grid, **shape)
                _check(sr, xf, off, form | STAGES[(grid + x_off + 1) % 4], x_off, grid=grid, **shape)
        _check(sr, xf, off, form | sr.LAST_BLOCK | 0x100, **shape)
        _check(sr, xf, off, form | sr.ATOMIC | 0x300, **shape)


@pytest.mark.parametrize("form", [0x4000, 0x8000])
@pytest.mark.parametrize("seg_len", [1, 3, 16, 64, 255, 268, 1000, 4097])
def test_warp_segments_equal_lengths(sr, seg_len, form):
    """Equal segments of every alignment against the 16/32-byte vectors (the
    head and tail elements take single loads) for the warp form, and against
    the element steps of the lane form; default shapes, every dtype."""
    nseg = max(1, (1 << 20) // seg_len)
    off = np.arange(nseg + 1, dtype=np.int64) * seg_len
    n = int(off[-1])
    for x_off in (0, 1, 2):
        _check(sr, workloads.uniform_i32(n, seed=seg_len), off, form, x_off)
        _check(sr, workloads.uniform_f32(n, seed=seg_len), off, form | sr.ATOMIC, x_off)
    x = workloads.lognormal_f32(n, seed=seg_len, sigma=2.0)
    bits = workloads.to_bf16_bits(x)
    dec_b = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
    codes, deq = workloads.to_e4m3_codes(x)
    od = torch.from_numpy(off).cuda()
    for x_off in (0, 1, 5):
        xd_b = _dev(bits.view(np.int16), x_off).view(torch.bfloat16)
        got = sr.reduce_sum_segmented(xd_b, od, variant=form).cpu().numpy()
        assert np.all(np.abs(got - oracle.segexact_f32(dec_b, off)) <=
                      4 * EPS32 * oracle.segsum_abs_f32(dec_b, off) + 1e-30), x_off
        xd_f = _dev(codes, x_off)
        got = sr.reduce_sum_segmented(xd_f, od, config=sr.make_config(form, scale=deq)).cpu().numpy()
        for s in range(0, nseg, max(1, nseg // 50)):
            a, b = off[s], off[s + 1]
            exs = oracle.to_float(oracle.exact_e4m3(codes[a:b], deq))
            assert abs(got[s] - exs) <= 4 * EPS32 * oracle.sum_e4m3(codes[a:b] & 0x7F, deq) * 1.001 + 1e-30


def test_warp_segments_plan_and_determinism(sr):
    r = sr.plan_segmented(1000, sr.F32, sr.make_config(sr.ATOMIC | WARP))
    assert r.variant & WARP and not r.variant & BULK and (r.vec_bytes, r.unroll) == (16, 2)
    r = sr.plan_segmented(1 << 20, sr.F32, sr.make_config(WARP))   # many segments: still no TMA form
    assert r.variant & WARP and not r.variant & BULK
    for other in (BULK, DENSE, LANE):
        with pytest.raises(sr.SRError) as e:
            sr.plan_segmented(1000, sr.F32, sr.make_config(sr.LAST_BLOCK | WARP | other))
        assert e.value.status == sr.ERR_UNSUPPORTED
    r = sr.plan_segmented(1 << 20, sr.F32, sr.make_config(LANE))
    assert r.variant & LANE and not r.variant & BULK and r.unroll == 4
    off = workloads.segment_offsets(3000, 1 << 22, seed=18, median=512, sigma=1.0, hi=1 << 16)
    xd, od = _dev(workloads.uniform_f32(int(off[-1]), seed=18)), torch.from_numpy(off).cuda()
    for form in (WARP, LANE):
        outs = [sr.reduce_sum_segmented(xd, od, variant=form | st).cpu().numpy() for st in STAGES]
        assert all(np.array_equal(outs[0], o) for o in outs[1:])   # same kernel, same order, any stage bits
        # captured once into a library-owned graph: replays give the same results
        out = torch.full((off.size - 1,), -1.0, dtype=torch.float32, device="cuda")
        g = sr.SegmentedGraph(xd, od, out, sr.make_config(form | sr.ATOMIC))
        for _ in range(3):
            out.fill_(-1.0)
            g.launch()
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), outs[0])
        g.close()
    assert sr.stream_status() == sr.OK


@pytest.mark.parametrize("stage", STAGES)
@pytest.mark.parametrize("flags", [0, BULK, WARP, LANE, ADAPT])
def test_checked_entry(sr, stage, flags):
    """sr_reduce_sum_segmented_checked: valid offsets give the oracle's sums;
    offsets past the declared element count, a decreasing pair or a negative
    first offset make the kernels read nothing and stream_status report
    SR_ERR_ARG, after which the stream works again.  The declared array sits
    inside padding, so even an unchecked read of these offsets stays in bounds."""
    n, nseg, pad = 200_000, 3000, 4096
    rng = np.random.default_rng(16)
    good = np.concatenate([[0], np.sort(rng.integers(0, n, nseg - 1)), [n]]).astype(np.int64)
    x = workloads.uniform_i32(n, seed=16)
    buf = torch.zeros(n + 2 * pad, dtype=torch.int32, device="cuda")
    buf[pad:pad + n] = torch.from_numpy(x).cuda()
    xd = buf[pad:pad + n]
    out = torch.empty(nseg, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    cfg = sr.make_config(stage | flags)

    def run(off):
        od = torch.from_numpy(off).cuda()
        out.fill_(-7)
        torch.cuda.synchronize()
        sr.check(sr.reduce_sum_segmented_checked_ptr(xd.data_ptr(), n, od.data_ptr(), nseg, sr.I32, out.data_ptr(),
                                                     cfg, s))
        s.synchronize()
        return sr.stream_status(s), out.cpu().numpy()
    st, got = run(good)
    assert st == sr.OK and np.array_equal(got, oracle.segsum_i32(x, good))
    past = good.copy()
    past[-1] = n + 1000                     # beyond the declared n, inside the padding
    swapped = good.copy()
    swapped[100], swapped[101] = good[101] + 1, good[100]   # a decreasing pair
    negative = good.copy()
    negative[0] = -8                        # before the array, inside the padding
    for bad in (past, swapped, negative):
        st, got = run(bad)
        assert st == sr.ERR_ARG
        assert np.all(got == (0 if stage == sr.ATOMIC and not flags & (WARP | LANE | ADAPT) else -7))  # nothing summed
    st, got = run(good)
    assert st == sr.OK and np.array_equal(got, oracle.segsum_i32(x, good))


# ---------------------------------------------------------------- adaptive form
@pytest.mark.parametrize("nseg,max_len", [(1, 0), (1, 1), (1, 100_000), (2, 5), (31, 0), (33, 7),
                                          (500, 300), (5000, 40), (300, 20_000), (40, 200_000)])
def test_adaptive_random_layouts(sr, nseg, max_len):
    """Random layouts through all three paths (segments of up to 512 bytes
    by lanes, up to one 16,384-element chunk by warps, longer ones queued as
    chunks), grids of one CTA up to the resident maximum, misaligned input."""
    off = workloads.random_segment_offsets(nseg, max_len, seed=nseg + max_len + 7)
    n = int(off[-1])
    xf = workloads.uniform_f32(n, seed=11)
    xi = workloads.uniform_i32(n, seed=11)
    for grid in (0, 1, 3):
        for x_off in (0, 1, 3):
            _check(sr, xi, off, ADAPT, x_off, grid=grid)
            _check(sr, xf, off, ADAPT, x_off, grid=grid)


@pytest.mark.parametrize("median,sigma,hi", [(40, 1.5, 1 << 16), (512, 2.5, 1 << 22), (4096, 1.94, 1 << 24)])
def test_adaptive_skewed_layouts(sr, median, sigma, hi):
    """Lognormal layouts with long tails (empty segments included): short,
    mid-length and multi-chunk segments in one call; int32 exact, binary32
    within the gate; the same result on every call (deterministic)."""
    n_total = 1 << 22
    nseg = max(1, n_total // (median * 2))
    off = workloads.segment_offsets(nseg, n_total, seed=median, median=median, sigma=sigma, lo=0, hi=hi)
    n = int(off[-1])
    xi = workloads.uniform_i32(n, seed=12)
    xf = workloads.uniform_f32(n, seed=12)
    _check(sr, xi, off, ADAPT)
    got = _check(sr, xf, off, ADAPT, 1)
    for _ in range(3):
        assert np.array_equal(_check(sr, xf, off, ADAPT, 1), got)


@pytest.mark.parametrize("flags", [0x100, 0x300, 0x200])
def test_adaptive_precision_flags(sr, flags):
    off = workloads.segment_offsets(600, 1 << 22, seed=13, median=1024, sigma=2.5, hi=1 << 21)
    x = workloads.lognormal_f32(int(off[-1]), seed=13, sigma=3.0)
    _check(sr, x, off, ADAPT | flags)


def test_adaptive_bf16_and_fp8(sr):
    off = workloads.segment_offsets(400, 1 << 21, seed=14, median=256, sigma=2.5, hi=1 << 20)
    n = int(off[-1])
    x = workloads.lognormal_f32(n, seed=14, sigma=2.0)
    bits = workloads.to_bf16_bits(x)
    codes, deq = workloads.to_e4m3_codes(x)
    od = torch.from_numpy(off).cuda()
    dec_b = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
    xd_b = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    got = sr.reduce_sum_segmented(xd_b, od, variant=ADAPT).cpu().numpy()
    ex = oracle.segexact_f32(dec_b, off)
    assert np.all(np.abs(got - ex) <= 4 * EPS32 * oracle.segsum_abs_f32(dec_b, off) + 1e-30)
    dec_f = (torch.from_numpy(codes).view(torch.float8_e4m3fn).float() * deq).numpy()
    got = sr.reduce_sum_segmented(torch.from_numpy(codes).cuda(), od,
                                  config=sr.make_config(ADAPT, scale=deq)).cpu().numpy()
    for s in range(400):
        a, b = off[s], off[s + 1]
        exs = oracle.to_float(oracle.exact_e4m3(codes[a:b], deq))
        sabs = float(np.abs(dec_f[a:b]).astype(np.float64).sum())
        assert abs(got[s] - exs) <= 4 * EPS32 * sabs * 1.001 + 1e-30, s


def test_adaptive_leaves_the_workspace_clean(sr):
    """The chunk queue lives in the stream's segmented workspace beside the
    flat split's tickets: after adaptive calls, last-block-done flat-split
    calls on the same stream (which need those tickets at zero) stay exact,
    and so does the next adaptive call."""
    off = workloads.segment_offsets(2000, 1 << 22, seed=15, median=2048, sigma=2.0, hi=1 << 20)
    x = workloads.uniform_i32(int(off[-1]), seed=15)
    for v in (ADAPT, 3, ADAPT, 3, 3 | BULK, ADAPT):
        _check(sr, x, off, v)
    assert sr.stream_status() == sr.OK


def test_adaptive_in_a_graph(sr):
    off = workloads.segment_offsets(3000, 1 << 22, seed=17, median=512, sigma=2.5, hi=1 << 20)
    x = workloads.uniform_f32(int(off[-1]), seed=17)
    xd, od = _dev(x), torch.from_numpy(off).cuda()
    out = torch.empty(3000, dtype=torch.float32, device="cuda")
    ref = sr.reduce_sum_segmented(xd, od, variant=ADAPT).cpu().numpy()
    g = sr.SegmentedGraph(xd, od, out, sr.make_config(ADAPT))
    for _ in range(3):
        out.fill_(-1)
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
    g.close()
    assert sr.stream_status() == sr.OK


def test_adaptive_refusals(sr):
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    od = torch.tensor([0, 32, 64], dtype=torch.int64, device="cuda")
    out = torch.empty(2, dtype=torch.float32, device="cuda")
    props = torch.cuda.get_device_properties(0)
    for kw, want in (({"vec_bytes": 32}, sr.ERR_UNSUPPORTED), ({"unroll": 4}, sr.ERR_UNSUPPORTED),
                     ({"block_threads": 128}, sr.ERR_UNSUPPORTED),
                     ({"grid": props.multi_processor_count * 40}, sr.ERR_LAUNCH)):  # valid, not co-resident
        st = sr.reduce_sum_segmented_ptr(x.data_ptr(), od.data_ptr(), 2, sr.F32, out.data_ptr(),
                                         sr.make_config(ADAPT, **kw))
        assert st == want, kw
    for other in (BULK, WARP, LANE, DENSE):
        st = sr.reduce_sum_segmented_ptr(x.data_ptr(), od.data_ptr(), 2, sr.F32, out.data_ptr(),
                                         sr.make_config(ADAPT | other))
        assert st == sr.ERR_UNSUPPORTED


@pytest.mark.slow
def test_adaptive_largest_queue(sr):
    """2^30 int32 values in ~32,000 segments of 16,385 to 50,000 elements:
    the chunk size grows past 16,384 elements (2 x 2^30 / 98,304 = 21,846)
    and the queue fills to ~80 % of its capacity; exact per segment."""
    rng = np.random.default_rng(18)
    lens = rng.integers(16_385, 50_001, 40_000)
    lens = lens[np.cumsum(lens) <= (1 << 30)]
    off = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    n = int(off[-1])
    xd = torch.randint(-1000, 1001, (n,), dtype=torch.int32, device="cuda")
    od = torch.from_numpy(off).cuda()
    got = sr.reduce_sum_segmented(xd, od, variant=ADAPT).cpu().numpy()
    x = xd.cpu().numpy()
    assert np.array_equal(got, oracle.segsum_i32(x, off))
    assert sr.stream_status() == sr.OK
