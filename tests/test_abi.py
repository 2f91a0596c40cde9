"""The C-ABI library builds, loads, exports every symbol include/*.h declares,
and rejects invalid calls before touching the GPU.  No GPU needed."""
import ctypes
import glob
import os
import re

import pytest

import paper_2004_05371_gb300 as sr
from paper_2004_05371_gb300 import build as sr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sr_build.build()
    return sr.load()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(sr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared_symbols()
    for required in ["sr_reduce_sum", "sr_reduce_sum_ex", "sr_stream_status", "sr_plan",
                     "sr_status_string", "sr_last_cuda_error", "sr_version"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for s in range(7):
        assert sr.status_string(s).startswith("SR_")


def _call(x, n, dtype, out, variant=0, **kw):
    c = sr.make_config(variant, **kw)
    return sr.reduce_sum_ptr(x, n, dtype, out, c, stream=0)


ALIGNED = 1 << 20   # stand-in device addresses: never dereferenced on the host


def test_rejects_bad_arguments_without_gpu(lib):
    assert _call(ALIGNED, -1, sr.F32, ALIGNED) == sr.ERR_ARG
    assert _call(0, 10, sr.F32, ALIGNED) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, 0) == sr.ERR_ARG
    assert _call(ALIGNED, 10, 7, ALIGNED) == sr.ERR_DTYPE
    assert _call(ALIGNED + 2, 10, sr.F32, ALIGNED) == sr.ERR_ARG        # misaligned x
    assert _call(ALIGNED, 10, sr.I32, ALIGNED + 4) == sr.ERR_ARG        # int64 out needs 8 B
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, variant=0x8000) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, variant=6) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, variant=sr.CLUSTER(5)) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, block_threads=48) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, vec_bytes=8) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, unroll=3) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, stages=9) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, tile_bytes=1000) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, grid=70000) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, scale=float("nan")) == sr.ERR_ARG
    assert _call(ALIGNED, 10, sr.F32, ALIGNED, variant=sr.GRID_SYNC | sr.CLUSTER(1)) == sr.ERR_UNSUPPORTED
    # BF16 input may start on any 2-byte boundary, FP8 on any byte
    assert _call(ALIGNED + 1, 10, sr.BF16, ALIGNED) == sr.ERR_ARG


def test_valid_call_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _call(ALIGNED, 10, sr.F32, ALIGNED) == sr.ERR_CUDA
    assert _call(ALIGNED + 1, 10, sr.FP8E4M3, ALIGNED) == sr.ERR_CUDA


def test_segmented_rejects_bad_arguments_without_gpu(lib):
    def call(nseg=4, dtype=sr.F32, x=ALIGNED, off=ALIGNED, out=ALIGNED, **kw):
        return sr.reduce_sum_segmented_ptr(x, off, nseg, dtype, out, sr.make_config(**kw), stream=0)
    assert call(nseg=-1) == sr.ERR_ARG
    assert call(x=0) == sr.ERR_ARG
    assert call(off=0) == sr.ERR_ARG
    assert call(out=0) == sr.ERR_ARG
    assert call(dtype=9) == sr.ERR_DTYPE
    assert call(off=ALIGNED + 4) == sr.ERR_ARG                     # offsets need 8-byte alignment
    assert call(dtype=sr.I32, out=ALIGNED + 4) == sr.ERR_ARG       # int64 results need 8 bytes
    assert call(variant=sr.SINGLE_CLUSTER) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.LAST_BLOCK | sr.F_BULK | sr.F_DENSE_SEGMENTS) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.LAST_BLOCK | sr.F_WARP_SEGMENTS | sr.F_BULK) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.ATOMIC | sr.F_WARP_SEGMENTS | sr.F_DENSE_SEGMENTS) == sr.ERR_UNSUPPORTED
    for other in (sr.F_BULK, sr.F_DENSE_SEGMENTS, sr.F_WARP_SEGMENTS):
        assert call(variant=sr.TWO_KERNEL | sr.F_LANE_SEGMENTS | other) == sr.ERR_UNSUPPORTED
    assert call(variant=sr.LAST_BLOCK | sr.F_BULK, unroll=1) == sr.ERR_ARG     # TMA chunks: 2, 4 or 8 rows
    assert call(variant=sr.LAST_BLOCK | sr.F_BULK, stages=9) == sr.ERR_ARG
    assert call(variant=sr.LAST_BLOCK | sr.CLUSTER(1)) == sr.ERR_UNSUPPORTED
    assert call(block_threads=100) == sr.ERR_ARG
    assert call(grid=100000, block_threads=512) == sr.ERR_ARG      # more than 65536 warps
    assert call(block_threads=1024) == sr.ERR_ARG                  # segmented CTAs: at most 512 threads
    assert call(nseg=0, x=0, off=0, out=0) == sr.OK                 # nothing to do, nothing launched


def test_differential_latency_host_code_matches_oracle(lib):
    """Eqs. 7-8 as computed by the library's host code vs the oracle's."""
    import numpy as np
    from oracle import model
    rng = np.random.default_rng(4)
    L1 = list(5000 + 3.5 * 1e5 + rng.normal(0, 30, 17))
    L2 = list(5000 + 3.5 * 1e4 + rng.normal(0, 20, 11))
    t, sg = sr.differential_latency(L1, L2, 100_000, 10_000)
    t_o, sg_o = model.differential_latency(L1, L2, 100_000, 10_000)
    assert t == pytest.approx(t_o, rel=1e-12) and sg == pytest.approx(sg_o, rel=1e-12)
    c = ctypes.c_double()
    arr = (ctypes.c_double * 1)(1.0)
    assert lib.sr_differential_latency(arr, 1, arr, 1, 2, 1, ctypes.byref(c), ctypes.byref(c)) == sr.ERR_ARG


def test_checked_segmented_rejects_bad_arguments_without_gpu(lib):
    def call(n_elems=16, x=ALIGNED, nseg=4, **kw):
        return sr.reduce_sum_segmented_checked_ptr(x, n_elems, ALIGNED, nseg, sr.F32, ALIGNED, sr.make_config(**kw),
                                                   stream=0)
    assert call(n_elems=-1) == sr.ERR_ARG
    assert call(x=0) == sr.ERR_ARG                       # data pointer required when n_elems > 0
    assert call(nseg=-1) == sr.ERR_ARG
    assert call(nseg=0) == sr.OK                         # nothing to check, nothing launched
    assert call(variant=sr.SINGLE_CLUSTER) == sr.ERR_UNSUPPORTED


def test_barrier_bench_rejects_bad_config_without_gpu(lib):
    def run(**kw):
        c = sr.BarrierConfig(**kw)
        r = sr.BarrierResult()
        return lib.sr_barrier_bench_ex(ctypes.byref(c), ctypes.byref(r))
    assert run(level=99) == sr.ERR_ARG
    assert run(level=sr.LEVEL_WARP, iters=5) == sr.ERR_ARG
    assert run(level=sr.LEVEL_WARP, group=3) == sr.ERR_ARG          # tiles are powers of two
    assert run(level=sr.LEVEL_COALESCED, group=33) == sr.ERR_ARG
    assert run(level=sr.LEVEL_BLOCK, threads=1000) == sr.ERR_ARG
    assert run(level=sr.LEVEL_CLUSTER, cluster=3) == sr.ERR_ARG
    assert run(level=sr.LEVEL_GRID, reps=1) == sr.ERR_ARG
    assert run(level=sr.LEVEL_WARP_REDUCE, method=7) == sr.ERR_ARG    # Table V has 7 methods
    assert run(level=sr.LEVEL_WARP_REDUCE, method=-1) == sr.ERR_ARG
    assert run(level=sr.LEVEL_WARP_REDUCE, method=sr.WR_FP32 | 7) == sr.ERR_ARG
    assert run(level=sr.LEVEL_WARP_REDUCE, method=32) == sr.ERR_ARG
    assert run(level=sr.LEVEL_KERNEL, method=3) == sr.ERR_ARG         # 3 launch functions
    assert run(level=sr.LEVEL_BLOCK, method=1) == sr.ERR_ARG          # no method elsewhere
    assert run(level=sr.LEVEL_KERNEL, method=sr.LAUNCH_CLUSTER, cluster=4, blocks=6) == sr.ERR_ARG
    assert run(level=sr.LEVEL_BLOCK, cluster=2) == sr.ERR_ARG
    assert lib.sr_barrier_bench_ex(None, None) == sr.ERR_ARG


def test_structs_match_the_header(tmp_path):
    """Every ctypes mirror has the layout the C compiler gives the header's
    struct: a C program built against include/sr.h prints sizeof and the
    offset of every field, which must equal the binding's."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"sr_config": sr.Config, "sr_barrier_config": sr.BarrierConfig,
               "sr_barrier_result": sr.BarrierResult, "sr_model_params": sr.ModelParams}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sr.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-x", "c", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                                 text=True).stdout.splitlines())
    for cname, py in mirrors.items():
        assert int(got[cname + " size"]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s %s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_candidate_set(lib):
    c40 = sr.candidates(152)
    assert len(c40) == 40
    c160 = sr.candidates(152, full=True)
    assert len(c160) == 160
    stages = {c.variant for c in c40}
    assert stages == {sr.TWO_KERNEL, sr.ATOMIC, sr.LAST_BLOCK, sr.GRID_SYNC}
    assert {c.grid for c in c40} == {8, 152, 304, 608, 1216}
    assert {c.vec_bytes for c in c40} == {16, 32} and {c.unroll for c in c160} == {1, 2, 4, 8}
    assert lib.sr_candidates(0, 0, None, 0) < 0


def test_analytic_selector_is_eq2(lib):
    """Two candidates that differ only in grid size: with the per-CTA cost as
    the extra synchronisation of the larger grid, the host selector's choice
    must equal Eq. 2 of the oracle's performance model for every N."""
    import numpy as np
    from oracle import model
    p = sr.ModelParams(sms=100, hbm_bytes_per_ns=5000.0, mem_latency_ns=800.0, launch_ns=0.0, grid_sync_ns=0.0,
                       last_block_ns=0.0, atomic_ns=0.0, per_cta_ns=3000.0, per_segment_ns=0.0)
    basic = sr.make_config(sr.LAST_BLOCK, grid=8, block_threads=256, vec_bytes=16, unroll=4)
    more = sr.make_config(sr.LAST_BLOCK, grid=800, block_threads=256, vec_bytes=16, unroll=4)
    cands = (sr.Config * 2)(basic, more)
    warp_bytes = 32 * 16 * 4
    thr_b = min(p.hbm_bytes_per_ns, 8 * 8 * warp_bytes / p.mem_latency_ns)
    thr_m = min(p.hbm_bytes_per_ns, 800 * 8 * warp_bytes / p.mem_latency_ns)
    t_sync = p.per_cta_ns * (800 - 8) / p.sms
    for N in np.geomspace(1e3, 1e9, 600):
        n = int(N) // 4
        i, _ = sr.select_analytic(p, n, sr.F32, 1, cands)
        assert (i == 0) == model.prefer_basic(n * 4, p.mem_latency_ns, t_sync, thr_b, thr_m), N


def test_host_entry_rejects_without_gpu(lib):
    import numpy as np
    x = np.zeros(16, np.float32)
    out = np.zeros(1, np.float64)
    xp, op = x.ctypes.data, out.ctypes.data
    assert sr.reduce_sum_host_ptr(xp, 16, sr.F32, 0, None, stream=0) == sr.ERR_ARG
    assert sr.reduce_sum_host_ptr(xp, -1, sr.F32, op, None, stream=0) == sr.ERR_ARG
    assert sr.reduce_sum_host_ptr(xp, 16, 8, op, None, stream=0) == sr.ERR_DTYPE
    assert sr.reduce_sum_host_ptr(xp, 16, sr.F32, op, sr.make_config(sr.ATOMIC), stream=0) == sr.ERR_UNSUPPORTED
    assert sr.reduce_sum_host_ptr(xp + 2, 4, sr.F32, op, None, stream=0) == sr.ERR_ARG


def test_segmented_layout_flags_without_gpu(lib):
    """The selected segmented path's form rule, a pure host function."""
    f = sr.segmented_layout_flags
    M = 1 << 20  # "many" segments (the whole-segment forms need 2^19 or more)
    # fewer segments: the dense kernel for uniformly short ones, else the plain form
    assert f(152, sr.F32, 20_000, 24.0, 0.0, 24.0) == sr.F_DENSE_SEGMENTS       # 96 bytes, uniform
    assert f(152, sr.F32, 20_000, 128.0, 64.0, 0.0) == sr.F_DENSE_SEGMENTS      # 512 bytes, std = mean / 2
    assert f(152, sr.F32, 20_000, 129.0, 0.0, 129.0) == 0                      # just over 512 bytes
    assert f(152, sr.FP8E4M3, 20_000, 512.0, 0.0, 512.0) == sr.F_DENSE_SEGMENTS  # bytes, not elements
    assert f(152, sr.F32, (1 << 19) - 1, 16.0, 0.0, 16.0) == sr.F_DENSE_SEGMENTS
    assert f(152, sr.F32, 10_000, 26843.5, 80000.0, 1 << 24) == 0               # the 10,000-segment batch
    # many uniform segments up to 1 KiB, none above 4x the mean: a thread each
    assert f(152, sr.F32, 1 << 24, 16.0, 0.0, 16.0) == sr.F_LANE_SEGMENTS
    assert f(152, sr.F32, 1 << 22, 64.0, 0.0, 64.0) == sr.F_LANE_SEGMENTS
    assert f(152, sr.F32, M, 128.0, 64.0, 256.0) == sr.F_LANE_SEGMENTS
    assert f(152, sr.BF16, M, 256.0, 0.0, 256.0) == sr.F_LANE_SEGMENTS
    assert f(152, sr.F32, M, 256.0, 0.0, 256.0) == sr.F_LANE_SEGMENTS          # 1 KiB
    assert f(152, sr.F32, M, 257.0, 0.0, 257.0) == sr.F_WARP_SEGMENTS          # just over 1 KiB
    assert f(152, sr.F32, 1 << 24, 16.0, 4.0, 65.0) == sr.F_DENSE_SEGMENTS     # one above 4x the mean
    assert f(152, sr.F32, M, 16.0, 9.0, 30.0) == sr.F_WARP_SEGMENTS            # spread: neither
    # many segments, no segment above twice a warp's share: a warp each
    assert f(152, sr.F32, 1_000_000, 268.0, 0.0, 268.0) == sr.F_WARP_SEGMENTS   # 1072 bytes
    assert f(152, sr.F32, (1 << 19) - 1, 268.0, 0.0, 268.0) == 0               # too few segments
    share = 268.0 * 1_000_000 / (32 * 152)
    assert f(152, sr.F32, 1_000_000, 268.0, 150.0, 2 * share) == sr.F_WARP_SEGMENTS
    assert f(152, sr.F32, 1_000_000, 268.0, 150.0, 2 * share + 1) == 0          # one segment too long
    assert f(152, sr.F32, 1_000_000, 268.0, 20000.0, 0.0) == sr.F_WARP_SEGMENTS  # unknown max: mean + 4 std
    assert f(152, sr.F32, 1_000_000, 268.0, 40000.0, 0.0) == 0
    for bad in ((0, sr.F32, 10, 1.0, 0.0, 1.0), (152, sr.F32, -1, 1.0, 0.0, 1.0),
                (152, sr.F32, 10, float("nan"), 0.0, 1.0), (152, sr.F32, 10, 1.0, -1.0, 1.0)):
        with pytest.raises(sr.SRError) as e:
            f(*bad)
        assert e.value.status == sr.ERR_ARG
    with pytest.raises(sr.SRError) as e:
        f(152, 7, 10, 1.0, 0.0, 1.0)
    assert e.value.status == sr.ERR_DTYPE
