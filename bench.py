#!/usr/bin/env python3
"""Throughput of the device-wide sum on GB300.

One step = one call of the library's reduction over the whole headline
workload: n = 2^28 binary32 values drawn U[-1, 1] (seed 0), 1 GiB, resident in
HBM before timing starts.  The input is larger than L2 (129 MB), so no flush is
needed between steps.  Prints one JSON line (rank 0).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (torchrun), every rank reduces its own copy of the workload on its
own GPU (independent replicas: the path has no exchange step on one box);
value = bytes reduced by all ranks / max-over-ranks time.
"""
import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Reduce GB/s & %HBM peak at 2^28 FP32; µs at 2^14; batched vs plain speedup"
N_HEADLINE = 1 << 28
N_LATENCY = 1 << 14
WORKLOAD = "device-wide sum, n=2^28 FP32 U[-1,1] seed 0 (1 GiB)"
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons.  Only samples
    whose timestamps fall inside [t_load0, t_load1] (host wall clock: the load
    window that encloses the timed region) are reported."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    @staticmethod
    def _ts(text):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text.strip(), fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self, t_load0, t_load1):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        rows = [[c.strip() for c in r.split(",")] for r in self.out.read().strip().splitlines()]
        rows = [r for r in rows if len(r) >= 10]
        inside = [r for r in rows if (self._ts(r[0]) or 0) >= t_load0 - 0.05 and (self._ts(r[0]) or 0) <= t_load1 + 0.05]
        use = inside or rows

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[2]) for r in use if num(r[2]) is not None]
        mx = [num(r[3]) for r in use if num(r[3]) is not None]
        pw = [num(r[4]) for r in use if num(r[4]) is not None]
        reasons = sorted({self.REASONS[i] for r in use for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "samples_in_load_window": len(inside),
                "power_w_max": max(pw) if pw else None,
                "window": "load window of back-to-back steps enclosing the timed region"}


# ---------------------------------------------------------- traffic record
KERNEL_SOURCES = ["sr_device.cuh", "sr_reduce_kernels.cuh", "sr_kparams.h", "sr_reduce_f32.cu"]


def kernel_source_hash():
    """Hash of the sources the single-array FP32 kernels are compiled from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2004_05371_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_tag):
    """DRAM bytes per launch from the committed ncu summary of this kernel,
    or None when the summary was taken on a different kernel source."""
    src = kernel_source_hash()
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(p) as f:
            text = f.read()
        m = re.search(r"traffic_record:\s*kernel=(\S+)\s+source=(\S+)\s+bytes_per_launch=(\d+)", text)
        if m and m.group(1) == kernel_tag and m.group(2) == src:
            return int(m.group(3))
    return None


# -------------------------------------------------------------- CPU baseline
def cpu_baseline(seconds=10.0):
    """The oracle (sequential FP64 loop, one host thread) on a bounded sample."""
    import numpy as np
    import oracle
    import workloads
    n = 1 << 25
    x = workloads.uniform_f32(n, seed=0)
    oracle.sum_f32(x[:1024])
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.sum_f32(x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    gbs = reps * n * 4 / el / 1e9
    return {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "%d passes of the sequential FP64 loop over the first 2^25 elements (128 MiB) of the "
                      "same U[-1,1] seed-0 workload, %.1f s" % (reps, el),
            "cpu": _cpu_model(), "host_cores": os.cpu_count(),
            "parallel": cpu_baseline_parallel(x, seconds / 2)}


def cpu_baseline_parallel(x, seconds):
    """The same oracle loop on every host core: the sample cut into one
    contiguous slice per thread (the C loop runs without the interpreter lock),
    the slices' FP64 partials added in slice order."""
    import concurrent.futures as cf
    import numpy as np
    import oracle
    T = max(1, os.cpu_count() or 1)
    n = x.size
    cuts = [n * i // T for i in range(T + 1)]
    parts = [x[cuts[i]:cuts[i + 1]] for i in range(T)]
    with cf.ThreadPoolExecutor(max_workers=T) as ex:
        def one_pass():
            return float(np.sum(np.array(list(ex.map(oracle.sum_f32, parts)), dtype=np.float64)))
        s_par = one_pass()
        reps, t0 = 0, time.perf_counter()
        while True:
            one_pass()
            reps += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                break
    s_seq = oracle.sum_f32(x)
    return {"value": round(reps * n * 4 / el / 1e9, 3), "unit": "GB/s", "cores": T,
            "sample": "%d passes over the same 2^25 elements, %d threads each running the sequential FP64 loop "
                      "on one contiguous slice, partials added in order, %.1f s" % (reps, T, el),
            "rel_diff_vs_sequential": abs(s_par - s_seq) / max(abs(s_seq), 1e-300)}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    per_step = []
    import oracle
    import workloads
    n = 1 << 25
    x = workloads.uniform_f32(n, seed=0)
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.sum_f32(x)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            per_step.append(dt)
    el = sum(per_step)
    gbs = args.steps * n * 4 / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * el / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "first 2^25 elements per step (the oracle is a "
                                                        "sequential CPU loop)", "l2": "input > L2"},
            "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "first 2^25 elements (128 MiB) of the workload per step"},
            "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", type=lambda s: int(s, 0), default=None,
                    help="explicit variant bits (default: the library's AUTO choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--n", type=int, default=N_HEADLINE, help="elements (profiling runs use a smaller case)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "fp8"],
                    help="input dtype of the timed loop (profiling runs of the precision path; the headline is f32)")
    ap.add_argument("--skip-extras", action="store_true", help="headline loop only (profiling runs)")
    ap.add_argument("--suite", default=None, choices=["selector", "barrier", "precision", "sweep", "segmented", "shapes", "seglayouts",
                             "latency"],
                    help="secondary measurement suites (JSON lines); the default run is the headline")
    ap.add_argument("--layout", default=None,
                    help="seglayouts suite: only the layouts whose name contains this text (profiling runs)")
    ap.add_argument("--shape-cases", default="all", choices=["all", "comp_mid", "gaps"],
                    help="shapes suite: every case, only the compensated 2-64 MiB ones, or only plain BF16 / "
                         "FP8 / int32 below 512 MiB and int32 above")
    ap.add_argument("--seg-form", default=None,
                    help="seglayouts suite: only these kernel forms and shapes, comma-separated (ldg256, dense256, "
                         "ldg512, dense512, tma, warp16, warp16u2, lane, lane32, adaptive)")
    ap.add_argument("--soak-seconds", type=float, default=0.5,
                    help="untimed back-to-back load before the timed region (clock sampling window)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    if args.impl == "reference":
        return run_reference(args)
    if args.suite:
        import bench_suites
        return bench_suites.run(args.suite, args)

    import numpy as np
    import torch
    import paper_2004_05371_gb300 as sr
    import workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sr.load()

    variant = sr.AUTO if args.variant is None else args.variant
    cfg = sr.make_config(variant)
    N = args.n
    DT = {"f32": sr.F32, "bf16": sr.BF16, "fp8": sr.FP8E4M3}[args.dtype]
    ES = {"f32": 4, "bf16": 2, "fp8": 1}[args.dtype]
    if DT == sr.FP8E4M3:
        cfg.scale = 1.0
    resolved = sr.plan(N, DT, cfg)
    stage = resolved.variant & sr.STAGE_MASK
    launches_per_step = 2 if stage == sr.TWO_KERNEL else 1

    x_host = workloads.uniform_f32(N, seed=0)
    if DT == sr.BF16:      # the same values rounded to BF16 / E4M3 (profiling runs)
        x = torch.from_numpy(workloads.to_bf16_bits(x_host).view(np.int16)).to(dev)
    elif DT == sr.FP8E4M3:
        x = torch.from_numpy(workloads.to_e4m3_codes(x_host, scale=448.0)[0]).to(dev)
    else:
        x = torch.from_numpy(x_host).to(dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step():
        sr.check(sr.reduce_sum_ptr(x.data_ptr(), N, DT, out.data_ptr(), cfg, sh))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # step duration estimate, to size a ~1 s load window around the timed region
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    soak_steps = int(args.soak_seconds / max(1e-6, e0.elapsed_time(e1) / 3e3))
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5 if args.soak_seconds > 0 else 0.0)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_load0 = time.time()
    for _ in range(soak_steps):        # untimed load before the timed region
        step()
    # the timed region: exactly K steps between two events on the launching
    # stream.  No event between launches: consecutive launches overlap their
    # set-up with the previous kernel's drain (programmatic dependent launch),
    # as they do in any stream of calls.
    t_start.record(stream)
    for i in range(args.steps):
        step()
    t_end.record(stream)
    for _ in range(soak_steps // 2):   # untimed load after it
        step()
    torch.cuda.synchronize()
    t_load1 = time.time()
    if pg:
        pg.barrier()
    clk = clocks.stop(t_load0, t_load1)
    elapsed_ms = t_start.elapsed_time(t_end)
    step_ms_local = elapsed_ms / args.steps
    if pg:
        t = torch.tensor([elapsed_ms], device=dev, dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    assert sr.stream_status(sh) == sr.OK

    bytes_step = N * ES
    value = ws * args.steps * bytes_step / (elapsed_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    # the dominant kernel's average launch duration: the timed region divided by
    # its K launches (one launch per step; a two-kernel step also counts its
    # one-CTA second kernel)
    kernel_ms = step_ms_local
    achieved = bytes_step / (kernel_ms * 1e-3) / 1e9
    if resolved.variant & sr.F_BULK:
        kernel_tag = "reduce_bulk_t%d_s%d" % (resolved.tile_bytes, resolved.stages)
    else:
        kernel_tag = "reduce_ldg_v%d_u%d" % (resolved.vec_bytes, resolved.unroll)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": recorded_traffic(kernel_tag),
                "peak_kind": "%s (MEASURED_PEAKS.json hbm_gbs, copy burst)" % peak_kind
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": kernel_tag, "algorithmic_bytes_per_launch": bytes_step,
                "per_launch_us": round(kernel_ms * 1e3, 2),
                "launch_timing": "CUDA events around the K timed steps on the launching stream / K"
                                 + (" (step = main kernel + one-CTA final kernel)" if launches_per_step == 2 else
                                    " (one launch per step)")}

    # ---- secondary: latency at 2^14 (device time per call inside a graph of calls)
    secondary, e2e = None, None
    if not args.skip_extras and DT == sr.F32:   # the secondary legs are FP32 by definition
        secondary = {}
        try:
            secondary["latency_2p14_us"] = latency_small(sr, torch, dev, stream)
        except Exception as e:  # reported, never hides the headline
            secondary["latency_2p14_error"] = str(e)[:200]
        try:
            secondary["library_reference"] = cub_reference(torch, x, N, stream, args)
        except Exception as e:
            secondary["library_reference_error"] = str(e)[:200]
        try:
            secondary["batched_vs_plain"] = batched_vs_plain(sr, torch, dev, stream)
        except Exception as e:
            secondary["batched_vs_plain_error"] = str(e)[:300]
        # ---- end to end: input in pinned host memory, copies inside the timed region
        try:
            e2e = end_to_end(sr, torch, dev, stream, x_host, args)
        except Exception as e:
            e2e = {"error": str(e)[:200]}
        if pg and e2e and "value" in e2e:
            t = torch.tensor([e2e["value"]], device=dev, dtype=torch.float64)
            pg.all_reduce(t, op=pg.ReduceOp.MIN)
            e2e["value"] = float(t.item()) * ws

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.skip_extras and DT == sr.F32:
        cpu = cpu_baseline(args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
                "data": "synthetic",
                "config": {"workload": WORKLOAD if (N == N_HEADLINE and DT == sr.F32) else "device-wide sum, n=%d %s U[-1,1] seed 0" % (N, args.dtype.upper()), "n": N, "variant": "0x%x" % resolved.variant,
                           "stage": sr.STAGE_NAMES.get(stage), "grid": resolved.grid,
                           "block": resolved.block_threads, "vec_bytes": resolved.vec_bytes,
                           "unroll": resolved.unroll, "tile_bytes": resolved.tile_bytes,
                           "stages": resolved.stages, "l2": "input (1 GiB) larger than L2: no flush",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "pct_hbm_peak": round(value / ws / peak, 4),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk, "secondary": secondary}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def latency_small(sr, torch, dev, stream, calls=1000):
    """Device time per call at n = 2^14 FP32 (SR_AUTO's choice) in a CUDA
    graph of `calls` back-to-back calls: warm (the same 64 KiB input every
    call, L2-resident), cold (each call after a 256 MiB write that evicts it
    from L2; the graph of the writes alone is timed and subtracted), CUB's
    DeviceReduce::Sum warm in the same protocol, and the host round trip of
    one call (launch, then stream synchronize)."""
    import libcmp
    import workloads
    x = torch.from_numpy(workloads.uniform_f32(N_LATENCY, seed=0)).to(dev)
    out = torch.empty((), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    cfg = sr.make_config(sr.AUTO)
    s = torch.cuda.Stream(dev)

    def graph_us(body, n_calls, reps=5):
        with torch.cuda.stream(s):
            for _ in range(3):
                body()      # the stream's first call allocates its workspace: before capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(n_calls):
                body()
        g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e3 / (reps * n_calls)

    def ours():
        sr.check(sr.reduce_sum_ptr(x.data_ptr(), N_LATENCY, sr.F32, out.data_ptr(), cfg,
                                   torch.cuda.current_stream().cuda_stream))
    warm = graph_us(ours, calls)
    cold_calls = 100
    flush_only = graph_us(lambda: flush.fill_(1), cold_calls)
    cold = graph_us(lambda: (flush.fill_(1), ours()), cold_calls) - flush_only
    cub = None
    try:
        libcmp.build()
        cmp = libcmp.lib()
        libcmp.check(cmp.cmp_prepare(N_LATENCY), "cmp_prepare")
        cub = graph_us(lambda: libcmp.check(cmp.cmp_cub_sum_f32(x.data_ptr(), N_LATENCY, out.data_ptr(),
                                                                torch.cuda.current_stream().cuda_stream), "cub"),
                       calls)
    except Exception:
        cub = None
    rt = []
    for _ in range(50):
        t0 = time.perf_counter()
        sr.check(sr.reduce_sum_ptr(x.data_ptr(), N_LATENCY, sr.F32, out.data_ptr(), cfg, stream.cuda_stream))
        stream.synchronize()
        rt.append((time.perf_counter() - t0) * 1e6)
    return {"graph_us_per_call": round(warm, 3), "calls": calls, "cold_us": round(cold, 3),
            "cold_protocol": "graph of %d (256 MiB write, call) pairs minus a graph of the writes alone" % cold_calls,
            "cub_us": None if cub is None else round(cub, 3),
            "host_roundtrip_us_median": round(statistics.median(rt), 2),
            "variant": "0x%x" % sr.plan(N_LATENCY, sr.F32, cfg).variant}


def segment_sums_f64(x, off):
    """Per-segment binary64 sums of x and of |x| for a CSR layout covering
    all of x (numpy; the accuracy figures of the segmented legs; the oracle
    stays out of the GPU arm).  Empty segments sum to 0."""
    import numpy as np
    assert int(off[-1]) == x.size
    lens = np.diff(off)
    nz = lens > 0
    starts = off[:-1][nz].astype(np.int64)
    x64 = x.astype(np.float64)
    s = np.zeros(lens.size)
    a = np.zeros(lens.size)
    if starts.size:
        # reduceat sums x[starts[k]:starts[k+1]] and x[starts[-1]:]: with the
        # empty segments left out these are exactly the non-empty segments
        s[nz] = np.add.reduceat(x64, starts)
        a[nz] = np.add.reduceat(np.abs(x64), starts)
    return s, a


def batched_vs_plain(sr, torch, dev, stream, nseg=10_000):
    """Batched segmented sum (10,000 lognormal segments, median 4096, sigma
    1.94, clipped to [1, 2^24], ~2^28 FP32 elements) in one graph-captured
    launch, against one plain sr_reduce_sum launch per segment (the plain
    launches timed both as a captured graph of 10,000 launches and eagerly)."""
    import numpy as np
    import workloads
    off = workloads.segment_offsets(nseg, 1 << 28, seed=0)
    n = int(off[-1])
    x_np = workloads.uniform_f32(n, seed=0)
    x = torch.from_numpy(x_np).to(dev)
    od = torch.from_numpy(off).to(dev)
    out_b = torch.empty(nseg, dtype=torch.float32, device=dev)
    out_p = torch.empty(nseg, dtype=torch.float32, device=dev)
    # the batched launch's tile (unroll), vector width, grid and grid stage come
    # from the exhaustive autotuner, run on this workload
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cands = sr.candidates(sms, full=True)
    us = sr.autotune(x.data_ptr(), n, sr.F32, out_b.data_ptr(), cands, reps=3, offsets_ptr=od.data_ptr(),
                     nseg=nseg, stream=stream)
    best = int(np.argmin(us))
    cfg = cands[best]
    sr.check(sr.reduce_sum_segmented_ptr(x.data_ptr(), od.data_ptr(), nseg, sr.F32, out_b.data_ptr(), cfg,
                                         stream.cuda_stream))
    g = sr.SegmentedGraph(x, od, out_b, cfg)

    def time_it(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    batched_ms = time_it(lambda: g.launch(stream), 20)
    dflt = sr.make_config(sr.AUTO)
    default_us = time_it(lambda: sr.check(sr.reduce_sum_segmented_ptr(x.data_ptr(), od.data_ptr(), nseg, sr.F32,
                                                                      out_p.data_ptr(), dflt, stream.cuda_stream)),
                         10) * 1e3
    xp, op = x.data_ptr(), out_p.data_ptr()
    lens = np.diff(off)
    plain_cfg = sr.make_config(sr.AUTO)
    sh = stream.cuda_stream

    def plain_eager():
        for s in range(nseg):
            sr.check(sr.reduce_sum_ptr(xp + int(off[s]) * 4, int(lens[s]), sr.F32, op + 4 * s, plain_cfg, sh))

    eager_ms = time_it(plain_eager, 2)
    # the same 10,000 launches captured once into a graph (no host launch cost)
    cs = torch.cuda.Stream(dev)
    with torch.cuda.stream(cs):
        for s in range(nseg):  # first call on this stream allocates its workspace: before capture
            sr.check(sr.reduce_sum_ptr(xp + int(off[s]) * 4, int(lens[s]), sr.F32, op + 4 * s, plain_cfg,
                                       cs.cuda_stream))
    cs.synchronize()
    pg_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pg_graph, stream=cs):
        for s in range(nseg):
            sr.check(sr.reduce_sum_ptr(xp + int(off[s]) * 4, int(lens[s]), sr.F32, op + 4 * s, plain_cfg,
                                       cs.cuda_stream))
    plain_graph_ms = time_it(lambda: pg_graph.replay(), 3)
    torch.cuda.synchronize()
    ref, sabs = segment_sums_f64(x_np, off)
    gate = 4 * 2.0 ** -23 * sabs
    err_b = float(np.max(np.abs(out_b.cpu().numpy() - ref) / gate))
    err_p = float(np.max(np.abs(out_p.cpu().numpy() - ref) / gate))
    g.close()
    try:
        selected = learned_selected(sr, torch, stream, x, od, off, nseg, ref, gate, plain_graph_ms, batched_ms)
    except Exception as e:  # reported, never hides the rest
        selected = {"error": str(e)[:300]}
    r = sr.plan_segmented(nseg, sr.F32, cfg)
    return {"n": n, "nseg": nseg, "batched_us": round(batched_ms * 1e3, 2),
            "batched_gbs": round(n * 4 / (batched_ms * 1e-3) / 1e9, 1),
            "plain_graph_us": round(plain_graph_ms * 1e3, 1), "plain_eager_us": round(eager_ms * 1e3, 1),
            "speedup_vs_plain_graph": round(plain_graph_ms / batched_ms, 2),
            "speedup_vs_plain_eager": round(eager_ms / batched_ms, 2),
            "max_err_over_gate_batched": round(err_b, 4), "max_err_over_gate_plain": round(err_p, 4),
            "learned_selected": selected,
            "batched_config": {"stage": sr.STAGE_NAMES.get(r.variant & sr.STAGE_MASK), "grid": r.grid,
                               "block": r.block_threads, "vec_bytes": r.vec_bytes, "unroll": r.unroll,
                               "chosen_by": "sr_autotune over %d candidates (%.0f us best, %.0f us default)"
                                            % (len(cands), us[best], default_us)}}


def learned_selected(sr, torch, stream, x, od, off, nseg, ref, gate, plain_graph_ms, batched_ms,
                     train_shapes=320):
    """The learned-selected form of the same segmented workload
    (sr_reduce_sum_segmented_selected): a selector trained in this run on
    exhaustive autotuner timings of random shapes (n <= 2^28), its choice for
    this workload, the first call's host cost (features, inference kernel,
    class read back, launch) and the device time of later calls (choice
    memoised), against the plain per-segment launches and the autotuned
    batched launch."""
    import numpy as np
    from paper_2004_05371_gb300 import selector
    import workloads
    sms = torch.cuda.get_device_properties(x.device).multi_processor_count
    cands = sr.candidates(sms)
    t0 = time.perf_counter()
    tr = workloads.selector_shapes(train_shapes, seed=101)
    for s in tr:
        s["n"] = min(s["n"], 1 << 28)
        s["nseg"] = min(s["nseg"], s["n"])
    off_tr = [workloads.shape_offsets(s, i) if s["nseg"] > 1 else None for i, s in enumerate(tr)]
    T = selector.collect_timings(tr, off_tr, cands)
    t_collect = time.perf_counter() - t0
    t1 = time.perf_counter()
    sel, _ = selector.train(selector.features(tr, off_tr), selector.soft_targets(T), steps=3000)
    t_train = time.perf_counter() - t1
    nat = sel.native(cands)
    lens = np.diff(off).astype(np.float64)
    out = torch.empty(nseg, dtype=torch.float32, device=x.device)
    sh = stream.cuda_stream

    def call():
        sr.check(sr.reduce_sum_segmented_selected_ptr(nat, x.data_ptr(), od.data_ptr(), nseg, sr.F32, out.data_ptr(),
                                                      lens.mean(), lens.std(), lens.max(), stream=sh))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    call()
    stream.synchronize()
    first_us = (time.perf_counter() - t2) * 1e6
    for _ in range(3):
        call()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(20):
        call()
    b.record(stream)
    torch.cuda.synchronize()
    sel_ms = a.elapsed_time(b) / 20
    err = float(np.max(np.abs(out.cpu().numpy() - ref) / gate))
    c = nat.choose(int(round(lens.mean() * nseg)), sr.F32, nseg, lens.mean(), lens.std(), lens.max())
    nat.close()
    return {"selected_us": round(sel_ms * 1e3, 2), "first_call_us": round(first_us, 1),
            "speedup_vs_plain_graph": round(plain_graph_ms / sel_ms, 2),
            "vs_autotuned_batched": round(sel_ms / batched_ms - 1.0, 4),
            "max_err_over_gate": round(err, 4),
            "choice": {"stage": sr.STAGE_NAMES.get(c.variant & sr.STAGE_MASK), "grid": c.grid,
                       "vec_bytes": c.vec_bytes},
            "selector": "MLP 9-64-64-40 trained in this run: %d shapes x %d candidates timed by sr_autotune "
                        "(%.1f s), 3000 Adam steps by the library's kernels (%.1f s)"
                        % (len(tr), len(cands), t_collect, t_train)}


def cub_reference(torch, x, n, stream, args):
    """CUB's DeviceReduce::Sum on the same resident input with the headline's
    protocol (K back-to-back calls between two events after W warm-ups): a
    library point of comparison, never on the library's path."""
    import libcmp
    libcmp.build()
    cmp = libcmp.lib()
    libcmp.check(cmp.cmp_prepare(n), "cmp_prepare")
    out = torch.empty((), dtype=torch.float32, device=x.device)
    sh = stream.cuda_stream

    def call():
        libcmp.check(cmp.cmp_cub_sum_f32(x.data_ptr(), n, out.data_ptr(), sh), "cmp_cub_sum_f32")
    for _ in range(max(3, args.warmup)):
        call()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        call()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    return {"cub_device_reduce_us": round(ms * 1e3, 2), "gbs": round(n * 4 / (ms * 1e-3) / 1e9, 1),
            "result": float(out.item())}


def end_to_end(sr, torch, dev, stream, x_host, args):
    """The same metric from HOST memory through the C ABI's host-buffer entry
    point (sr_reduce_sum_host): every step copies the 1 GiB input from pinned
    host memory to the device (chunked, overlapped with the reduction) and
    reads the 4-byte result back.  Host wall clock around whole calls; the
    median of three blocks of k calls."""
    n = x_host.size
    pinned = torch.from_numpy(x_host).pin_memory()
    res = torch.zeros((), dtype=torch.float32).pin_memory()
    cfg = sr.make_config(sr.AUTO)
    sh = stream.cuda_stream

    def step():
        sr.check(sr.reduce_sum_host_ptr(pinned.data_ptr(), n, sr.F32, res.data_ptr(), cfg, sh))

    for _ in range(2):
        step()
    k = max(3, min(args.steps, 10))

    def timed_blocks(fn):
        # median over three blocks of k calls: one block disturbed by other
        # traffic on the shared host link does not set the number
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            for _ in range(k):
                fn()
            ts.append((time.perf_counter() - t0) / k)
        return statistics.median(ts)
    dt = timed_blocks(step)
    # the same call reading the pinned array in place over the CPU-GPU link
    direct = None
    dcfg = sr.make_config(sr.F_HOST_DIRECT)
    if sr.reduce_sum_host_ptr(pinned.data_ptr(), n, sr.F32, res.data_ptr(), dcfg, sh) == sr.OK:
        ddt = timed_blocks(lambda: sr.check(sr.reduce_sum_host_ptr(pinned.data_ptr(), n, sr.F32, res.data_ptr(),
                                                                    dcfg, sh)))
        direct = {"gbs": round(n * 4 / ddt / 1e9, 2), "ms_per_step": round(ddt * 1e3, 3),
                  "path": "sr_reduce_sum_host with SR_F_HOST_DIRECT (kernel reads pinned host memory in place)"}
    raw = raw_h2d_bound(torch, dev, pinned, timed_blocks)
    return {"value": round(n * 4 / dt / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": n * 4,
            "raw_h2d_gbs": raw, "value_over_raw_h2d": round((n * 4 / dt / 1e9) / max(raw.values()), 4),
            "d2h_bytes_per_step": 4, "ms_per_step": round(dt * 1e3, 3), "result": float(res.item()),
            "path": "sr_reduce_sum_host: pinned host input, 64 MiB chunks on two copy streams overlapped "
                    "with the chunk reductions, final combine, 4-byte read-back", "direct_read": direct}


def raw_h2d_bound(torch, dev, pinned, timed_blocks):
    """The host link's own figure for the same bytes: the pinned 1 GiB input
    copied to the device with no reduction, as one cudaMemcpyAsync and split
    into 2 and 4 chunks on as many streams (one cudaMemcpyAsync per chunk),
    host wall clock around copy + synchronize, as the e2e steps are timed."""
    nbytes = pinned.numel() * pinned.element_size()
    dst = torch.empty(pinned.numel(), dtype=pinned.dtype, device=dev)
    res = {}
    for k in (1, 2, 4):
        streams = [torch.cuda.Stream(dev) for _ in range(k)]
        step = (pinned.numel() + k - 1) // k

        def copy():
            for i, st in enumerate(streams):
                with torch.cuda.stream(st):
                    dst[i * step:(i + 1) * step].copy_(pinned[i * step:(i + 1) * step], non_blocking=True)
            for st in streams:
                st.synchronize()
        copy()
        res["streams_%d" % k] = round(nbytes / timed_blocks(copy) / 1e9, 2)
    del dst
    return res


if __name__ == "__main__":
    sys.exit(main())
