"""Parity of the CUDA reduction (through the C ABI) with the CPU oracle.

int32 input: bit-exact against the int64 sequential sum.
binary32 input: |S_gpu - S_exact| <= 4 * eps32 * sum|x| (eps32 = 2^-23), the
stated gate for the plain FP32 tree, on every input including same-sign
data, and <= gamma_m * sum|x| (Higham) with m the longest chain of additions
of the launch shape actually used.
Integer-valued binary32 arrays whose partial sums stay below 2^24 are exact
in any order, so there the result must equal the exact sum.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

STAGES = {"two_kernel": 1, "atomic": 2, "last_block": 3, "grid_sync": 4, "single_cluster": 5}
SIZES = [0, 1, 2, 3, 31, 32, 33, 127, 128, 129, 1023, 1025, 4099, (1 << 16) + 5, (1 << 20) + 3]
OFFSETS = [0, 1, 2, 3]


def _variants(sr):
    out = []
    for name, st in STAGES.items():
        for log2c in ([0] if st == sr.GRID_SYNC else [0, 1, 2, 3, 4]):
            for bulk in (False, True):
                out.append((name, st | sr.CLUSTER(log2c) | (sr.F_BULK if bulk else 0)))
    return out


def _to_dev(a: np.ndarray, offset: int):
    """Device copy of `a` starting `offset` elements past a 256-byte boundary."""
    buf = torch.zeros(a.size + offset + 8, dtype=torch.from_numpy(a[:0]).dtype, device="cuda")
    view = buf[offset:offset + a.size]
    if a.size:
        view.copy_(torch.from_numpy(a))
    return view


def _chain_bound(sr, n, dtype, variant, sum_abs):
    cfg = sr.plan(n, dtype, sr.make_config(variant))
    threads = max(1, cfg.grid * cfg.block_threads // 2)
    m = math.ceil(n / threads) * 4 + 64 + cfg.grid
    return oracle.gamma(m) * sum_abs


def _check_f32(sr, x_np, got, variant, exact=None, stated=True):
    """`stated`: also assert the 4*eps32*sum|x| gate (every tree form meets it
    on any data: the thread stage is blocked, no chain of additions longer
    than ~16); the launch-shape Higham bound is asserted everywhere."""
    exact = oracle.exact_f32(x_np) if exact is None else exact
    sabs = oracle.sum_abs_f32(x_np)
    err = abs(got - oracle.to_float(exact))
    if stated:
        assert err <= oracle.stated_fp32_bound(sabs), (got, oracle.to_float(exact), err)
    assert err <= _chain_bound(sr, x_np.size, sr.F32, variant, sabs) + 1e-300, (got, err)


@pytest.mark.parametrize("vname,variant", [pytest.param(n, v, id="%s-%x" % (n, v)) for n, v in
                                           _variants(__import__("paper_2004_05371_gb300"))])
def test_parity_sizes_offsets(sr, vname, variant):
    for n in SIZES:
        xf = workloads.uniform_f32(n, seed=n)
        xi = workloads.uniform_i32(n, seed=n)
        ref_i = oracle.sum_i32(xi)
        exact_f = oracle.exact_f32(xf)
        for off in OFFSETS:
            got_f = float(sr.reduce_sum(_to_dev(xf, off), variant=variant).item())
            _check_f32(sr, xf, got_f, variant, exact_f)
            got_i = int(sr.reduce_sum(_to_dev(xi, off), variant=variant).item())
            assert got_i == ref_i, (n, off, got_i, ref_i)
    torch.cuda.synchronize()
    assert sr.stream_status() == sr.OK


@pytest.mark.parametrize("vec", [16, 32])
@pytest.mark.parametrize("unroll", [1, 2, 4, 8])
@pytest.mark.parametrize("block", [32, 256, 1024])
def test_ldg_launch_shapes(sr, vec, unroll, block):
    n = (1 << 18) + 7
    xf = workloads.uniform_f32(n, seed=1)
    xi = workloads.uniform_i32(n, seed=1)
    exact_f, ref_i = oracle.exact_f32(xf), oracle.sum_i32(xi)
    for stage in (sr.TWO_KERNEL, sr.LAST_BLOCK, sr.GRID_SYNC):
        for off in (0, 3):
            cfg = sr.make_config(stage, vec_bytes=vec, unroll=unroll, block_threads=block)
            _check_f32(sr, xf, float(sr.reduce_sum(_to_dev(xf, off), config=cfg).item()), stage, exact_f)
            assert int(sr.reduce_sum(_to_dev(xi, off), config=cfg).item()) == ref_i


@pytest.mark.parametrize("tile,stages,block", [(1024, 2, 64), (4096, 3, 96), (16384, 4, 288),
                                               (32768, 6, 288), (65536, 3, 544), (229376 // 2, 2, 1024)])
def test_bulk_ring_shapes(sr, tile, stages, block):
    n = (1 << 20) + 13
    xf = workloads.uniform_f32(n, seed=2)
    xi = workloads.uniform_i32(n, seed=2)
    exact_f, ref_i = oracle.exact_f32(xf), oracle.sum_i32(xi)
    for stage in (sr.TWO_KERNEL, sr.LAST_BLOCK, sr.ATOMIC):
        for off in (0, 1):
            cfg = sr.make_config(stage | sr.F_BULK, tile_bytes=tile, stages=stages, block_threads=block)
            _check_f32(sr, xf, float(sr.reduce_sum(_to_dev(xf, off), config=cfg).item()), stage, exact_f)
            assert int(sr.reduce_sum(_to_dev(xi, off), config=cfg).item()) == ref_i
    torch.cuda.synchronize()
    assert sr.stream_status() == sr.OK


@pytest.mark.parametrize("grid", [1, 2, 7, 152, 999])
def test_explicit_grids(sr, grid):
    n = 300_001
    xf = workloads.uniform_f32(n, seed=3)
    xi = workloads.uniform_i32(n, seed=3)
    exact_f, ref_i = oracle.exact_f32(xf), oracle.sum_i32(xi)
    for stage in (sr.TWO_KERNEL, sr.ATOMIC, sr.LAST_BLOCK):
        for flags in (0, sr.F_BULK):
            cfg = sr.make_config(stage | flags, grid=grid)
            _check_f32(sr, xf, float(sr.reduce_sum(_to_dev(xf, 0), config=cfg).item()), stage, exact_f)
            assert int(sr.reduce_sum(_to_dev(xi, 0), config=cfg).item()) == ref_i


def test_closed_forms(sr):
    for n in [1, 1000, 65535, 65536, 65537, 1 << 20, (1 << 24) + 1]:
        x = np.arange(1, n + 1, dtype=np.int32)
        for stage in STAGES.values():
            assert int(sr.reduce_sum(_to_dev(x, 1), variant=stage).item()) == n * (n + 1) // 2
    n = 4096  # every partial sum is an integer below 2^24: exact in any order
    x = np.arange(1, n + 1, dtype=np.float32)
    for stage in STAGES.values():
        assert float(sr.reduce_sum(_to_dev(x, 2), variant=stage).item()) == n * (n + 1) / 2


def test_integer_valued_float_invariant(sr):
    n = 1 << 22
    cases = [np.ones(n, np.float32),
             np.tile(np.array([1.0, -1.0], np.float32), n // 2),
             np.append(np.tile(np.array([1.0, -1.0], np.float32), n // 2), np.float32(1.0)),
             np.tile(np.array([2.0 ** -3, -(2.0 ** -3)], np.float32), n // 2),
             np.full(1 << 24, 1.0, np.float32)]
    for x in cases:
        exact = oracle.to_float(oracle.exact_f32(x))
        for name, st in STAGES.items():
            for flags in (0, sr.F_BULK):
                got = float(sr.reduce_sum(_to_dev(x, 0), variant=st | flags).item())
                assert got == exact, (name, flags, got, exact)


# Every form whose grid stage is a tree (all but the atomic finish).
TREE_FORMS = {"auto": 0, "two_kernel": 1, "last_block": 3, "grid_sync": 4, "single_cluster": 5,
              "last_block_ring": 3 | 0x400, "last_block_cluster2": 3 | 0x10, "two_kernel_cluster4": 1 | 0x20}


@pytest.mark.slow
@pytest.mark.parametrize("n", [1 << 24, 1 << 28])
def test_same_sign_stated_gate(sr, n):
    """Same-sign data, where rounding errors do not cancel: constant 0.1f
    (exact sum n * fl32(0.1), n a power of two) and all-positive lognormal
    (sigma 4) magnitudes.  Every tree form meets the stated gate
    |err| <= 4 eps32 sum|x|.  The atomic finish adds its P unit partials one
    after another in arbitrary order, a chain of P additions on data whose
    partials are all alike, so there only the Higham bound of that chain is
    asserted (and the error is reported)."""
    c = np.float32(0.1)
    x = np.full(n, c, np.float32)
    exact = n * float(c)  # exact in binary64: n is a power of two
    d = _to_dev(x, 0)
    gate = oracle.stated_fp32_bound(exact)
    for name, v in TREE_FORMS.items():
        got = float(sr.reduce_sum(d, variant=v).item())
        assert abs(got - exact) <= gate, (name, got, exact, abs(got - exact) / gate)
    got = float(sr.reduce_sum(d, variant=sr.ATOMIC).item())
    assert abs(got - exact) <= _chain_bound(sr, n, sr.F32, sr.ATOMIC, exact), (got, exact)
    del d
    x = np.abs(workloads.lognormal_f32(n, seed=7))
    ex = oracle.to_float(oracle.exact_f32(x))
    sabs = oracle.sum_abs_f32(x)
    d = _to_dev(x, 0)
    for name, v in TREE_FORMS.items():
        got = float(sr.reduce_sum(d, variant=v).item())
        assert abs(got - ex) <= oracle.stated_fp32_bound(sabs), (name, got, ex)
    got = float(sr.reduce_sum(d, variant=sr.ATOMIC).item())
    assert abs(got - ex) <= _chain_bound(sr, n, sr.F32, sr.ATOMIC, sabs), (got, ex)
    del d
    torch.cuda.empty_cache()
    assert sr.stream_status() == sr.OK


def test_long_thread_chains_stay_blocked(sr):
    """One CTA over 2^22 constant values (8,192 values per word accumulator of
    each thread): the blocked thread stage keeps the error inside the stated
    gate on the LDG path and on a TMA ring whose tile gives each lane more
    than one block (64 KiB tiles, one consumer warp: 128 chunks per lane)."""
    n = 1 << 22
    c = np.float32(0.1)
    d = _to_dev(np.full(n, c, np.float32), 0)
    exact = n * float(c)
    gate = oracle.stated_fp32_bound(exact)
    for cfg in (sr.make_config(sr.SINGLE_CLUSTER, block_threads=128, vec_bytes=16, unroll=1),
                sr.make_config(sr.SINGLE_CLUSTER, block_threads=32, vec_bytes=32, unroll=8),
                sr.make_config(sr.LAST_BLOCK | sr.F_BULK, grid=1, block_threads=64, tile_bytes=65536, stages=2),
                sr.make_config(sr.TWO_KERNEL | sr.F_BULK, grid=3, block_threads=96, tile_bytes=32768, stages=3)):
        got = float(sr.reduce_sum(d, config=cfg).item())
        assert abs(got - exact) <= gate, (cfg.as_dict(), got, exact, abs(got - exact) / gate)
    for dt_name in ("bf16", "fp8"):
        if dt_name == "bf16":
            bits = workloads.to_bf16_bits(np.full(n, c, np.float32))
            xd = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
            v = float(np.frombuffer((bits[:1].astype(np.uint32) << 16).tobytes(), dtype=np.float32)[0])
            scale = None
        else:
            codes, scale = workloads.to_e4m3_codes(np.full(n, c, np.float32))
            xd = torch.from_numpy(codes).cuda()
            v = oracle.decode_e4m3(int(codes[0])) * scale
        ex = n * v
        for cfg in (sr.make_config(sr.SINGLE_CLUSTER, block_threads=128, vec_bytes=16, unroll=2,
                                   scale=scale or 0.0),
                    sr.make_config(sr.LAST_BLOCK | sr.F_BULK, grid=1, block_threads=64, tile_bytes=65536,
                                   stages=2, scale=scale or 0.0)):
            got = float(sr.reduce_sum(xd, config=cfg).item())
            assert abs(got - ex) <= oracle.stated_fp32_bound(abs(ex)), (dt_name, cfg.as_dict(), got, ex)


def test_int_extremes_and_permutation(sr):
    n = 1 << 26
    x = np.full(n, 2 ** 31 - 1, np.int32)
    for st in STAGES.values():
        assert int(sr.reduce_sum(_to_dev(x, 0), variant=st).item()) == n * (2 ** 31 - 1)
    x = np.full(n, -(2 ** 31), np.int32)
    assert int(sr.reduce_sum(_to_dev(x, 0), variant=sr.LAST_BLOCK).item()) == -n * 2 ** 31
    xi = workloads.uniform_i32(1 << 22, seed=0)
    p = np.random.default_rng(1).permutation(xi.size)
    for st in STAGES.values():
        a = int(sr.reduce_sum(_to_dev(xi, 0), variant=st).item())
        b = int(sr.reduce_sum(_to_dev(xi[p], 0), variant=st).item())
        assert a == b == oracle.sum_i32(xi)


def test_deterministic_stages_are_bitwise_repeatable(sr):
    x = _to_dev(workloads.uniform_f32(1 << 22, seed=5), 0)
    for st in (sr.TWO_KERNEL, sr.LAST_BLOCK, sr.GRID_SYNC, sr.SINGLE_CLUSTER):
        vals = {float(sr.reduce_sum(x, variant=st).item()) for _ in range(5)}
        assert len(vals) == 1, (st, vals)


def test_grid_sync_rejects_non_coresident_grid(sr):
    props = torch.cuda.get_device_properties(0)
    x = _to_dev(workloads.uniform_f32(1 << 16, seed=0), 0)
    out = torch.empty((), dtype=torch.float32, device="cuda")
    cfg = sr.make_config(sr.GRID_SYNC, grid=props.multi_processor_count * 64, block_threads=1024)
    st = sr.reduce_sum_ptr(x.data_ptr(), x.numel(), sr.F32, out.data_ptr(), cfg)
    assert st == sr.ERR_LAUNCH


def test_two_streams_have_separate_workspaces(sr):
    xa = workloads.uniform_i32(1 << 22, seed=10)
    xb = workloads.uniform_i32(1 << 22, seed=11)
    da, db = _to_dev(xa, 0), _to_dev(xb, 0)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    outs_a, outs_b = [], []
    for _ in range(20):
        with torch.cuda.stream(sa):
            outs_a.append(sr.reduce_sum(da, variant=sr.LAST_BLOCK, stream=sa))
        with torch.cuda.stream(sb):
            outs_b.append(sr.reduce_sum(db, variant=sr.LAST_BLOCK, stream=sb))
    torch.cuda.synchronize()
    assert all(int(o.item()) == oracle.sum_i32(xa) for o in outs_a)
    assert all(int(o.item()) == oracle.sum_i32(xb) for o in outs_b)
    assert sr.stream_status(sa) == sr.OK and sr.stream_status(sb) == sr.OK


@pytest.mark.slow
@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_full_size_2p28(sr, dtype):
    """The headline size (2^28 elements) in the default (AUTO) configuration
    and in every explicit grid stage."""
    n = 1 << 28
    if dtype == "f32":
        x = workloads.uniform_f32(n, seed=0)
        exact = oracle.exact_f32(x)
        d = _to_dev(x, 0)
        for st in (sr.AUTO, sr.TWO_KERNEL, sr.ATOMIC, sr.LAST_BLOCK, sr.GRID_SYNC,
                   sr.LAST_BLOCK | sr.F_BULK, sr.LAST_BLOCK | sr.CLUSTER(2)):
            _check_f32(sr, x, float(sr.reduce_sum(d, variant=st).item()), st, exact)
    else:
        x = workloads.uniform_i32(n, seed=0)
        ref = oracle.sum_i32(x)
        d = _to_dev(x, 0)
        for st in (sr.AUTO, sr.TWO_KERNEL, sr.ATOMIC, sr.LAST_BLOCK, sr.GRID_SYNC,
                   sr.LAST_BLOCK | sr.F_BULK, sr.LAST_BLOCK | sr.CLUSTER(2)):
            assert int(sr.reduce_sum(d, variant=st).item()) == ref


@pytest.mark.slow
def test_max_size_2p30_int32_worst_case(sr):
    """Largest size of the sweep: 2^30 int32 at INT32_MAX (sum 2^61 - 2^30)."""
    n = 1 << 30
    d = torch.full((n,), 2 ** 31 - 1, dtype=torch.int32, device="cuda")
    for st in (sr.LAST_BLOCK, sr.TWO_KERNEL, sr.LAST_BLOCK | sr.F_BULK):
        assert int(sr.reduce_sum(d, variant=st).item()) == n * (2 ** 31 - 1)
    del d
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_full_size_2p30_f32(sr):
    """The largest size of the sweep in binary32: 2^30 U[-1,1] values (4 GiB)
    through SR_AUTO (the TMA ring), the ring explicitly and the two-kernel
    form, against the exact sum."""
    n = 1 << 30
    x = workloads.uniform_f32(n, seed=30)
    exact = oracle.exact_f32(x)
    d = _to_dev(x, 0)
    for st in (sr.AUTO, sr.LAST_BLOCK | sr.F_BULK, sr.TWO_KERNEL):
        _check_f32(sr, x, float(sr.reduce_sum(d, variant=st).item()), st, exact)
    del d, x
    torch.cuda.empty_cache()
    assert sr.stream_status() == sr.OK


@pytest.mark.slow
def test_cluster_forms_2p26(sr):
    """Clusters of 4 CTAs (DSMEM merge) at 2^26 elements, above the sizes of
    the per-shape sweep: last-block-done and two-kernel finishes, LDG and the
    TMA ring, FP32 within the gates and int32 exactly."""
    n = (1 << 26) + 7
    xf = workloads.uniform_f32(n, seed=26)
    xi = workloads.uniform_i32(n, seed=26)
    exact_f, ref_i = oracle.exact_f32(xf), oracle.sum_i32(xi)
    df, di = _to_dev(xf, 1), _to_dev(xi, 1)
    for st in (sr.LAST_BLOCK, sr.TWO_KERNEL):
        for flags in (0, sr.F_BULK):
            v = st | sr.CLUSTER(2) | flags
            _check_f32(sr, xf, float(sr.reduce_sum(df, variant=v).item()), v, exact_f)
            assert int(sr.reduce_sum(di, variant=v).item()) == ref_i, hex(v)
    assert sr.stream_status() == sr.OK


@pytest.mark.slow
def test_auto_regime_boundaries(sr):
    """SR_AUTO on both sides of each of its size thresholds (16 KiB one CTA,
    1 MiB one cluster, 64 MiB two-kernel with 32-byte loads, 512 MiB two-kernel
    with 16-byte loads, above: TMA ring or per-dtype LDG) for every dtype,
    aligned and misaligned: int32 bit-exact, floating point within the gates."""
    for bound in (16 << 10, 1 << 20, 64 << 20, 512 << 20):
        big = bound == 512 << 20
        for dt, es in ((sr.F32, 4), (sr.I32, 4), (sr.BF16, 2), (sr.FP8E4M3, 1)):
            for d, off in (((1, 1),) if big else ((0, 0), (1, 1), (-1, 3))):
                n = bound // es + d
                seed = n % 1000
                if dt == sr.I32:
                    x = workloads.uniform_i32(n, seed=seed)
                    got = int(sr.reduce_sum(_to_dev(x, off)).item())
                    assert got == oracle.sum_i32(x), (bound, d, off)
                elif dt == sr.F32:
                    x = workloads.uniform_f32(n, seed=seed)
                    got = float(sr.reduce_sum(_to_dev(x, off)).item())
                    _check_f32(sr, x, got, sr.AUTO)
                elif dt == sr.BF16:
                    bits = workloads.to_bf16_bits(workloads.uniform_f32(n, seed=seed))
                    buf = np.zeros(n + off, np.uint16)
                    buf[off:] = bits
                    xd = torch.from_numpy(buf.view(np.int16)).cuda().view(torch.bfloat16)[off:]
                    got = float(sr.reduce_sum(xd).item())
                    dec = np.frombuffer((bits.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
                    ex = oracle.to_float(oracle.exact_bf16(bits))
                    assert abs(got - ex) <= oracle.stated_fp32_bound(oracle.sum_abs_f32(dec)), (bound, d, off)
                else:
                    codes, deq = workloads.to_e4m3_codes(workloads.uniform_f32(n, seed=seed))
                    buf = np.zeros(n + off, np.uint8)
                    buf[off:] = codes
                    xd = torch.from_numpy(buf).cuda()[off:]
                    got = float(sr.reduce_sum(xd, scale=deq).item())
                    ex = oracle.to_float(oracle.exact_e4m3(codes, deq))
                    assert abs(got - ex) <= oracle.stated_fp32_bound(oracle.sum_e4m3(codes & 0x7F, deq)), (bound, d)
                torch.cuda.empty_cache()
    assert sr.stream_status() == sr.OK
