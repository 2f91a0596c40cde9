"""Secondary measurement suites of bench.py (one JSON line per measurement).

  selector  : learned selector vs performance-model selector vs exhaustive
              autotuning on held-out random shapes (regret), training from
              ~20,000 autotuner timings
  barrier   : synchronisation cost per level and shape (Section V / IX)
  precision : 2^28-element lognormal / cancelling inputs in FP32, BF16 and FP8 (SR_AUTO),
              plain vs compensated vs compensated + FP64 combine: error against
              the exact sum and the FP64 oracle, and throughput
  sweep     : size sweep 2^10..2^30 for FP32 and int32, every grid stage
  segmented : the batched segmented workload in one graph launch per step
  shapes    : warm / cold launch-shape sweeps per dtype and size (the basis of
              SR_AUTO's table), SR_AUTO and CUB beside them
  seglayouts: the segmented kernel over sparse to dense segment layouts, with and
              without SR_F_DENSE_SEGMENTS
"""
import json
import math
import time

import numpy as np


def _emit(d):
    print(json.dumps(d), flush=True)


def _time_calls(torch, fn, reps, stream):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def selector_suite(args):
    import torch
    import paper_2004_05371_gb300 as sr
    from paper_2004_05371_gb300 import selector
    import workloads
    sr.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cands = sr.candidates(sms)
    t0 = time.time()
    tr = workloads.selector_shapes(500, seed=101)
    te = workloads.selector_shapes(1000, seed=202)
    off_tr = [workloads.shape_offsets(s, i) if s["nseg"] > 1 else None for i, s in enumerate(tr)]
    off_te = [workloads.shape_offsets(s, 50_000 + i) if s["nseg"] > 1 else None for i, s in enumerate(te)]
    Ttr = selector.collect_timings(tr, off_tr, cands)
    Tte = selector.collect_timings(te, off_te, cands)
    t_collect = time.time() - t0
    Xtr, Xte = selector.features(tr, off_tr), selector.features(te, off_te)
    t1 = time.time()
    sel, losses = selector.train(Xtr, selector.soft_targets(Ttr), steps=4000, lr=3e-3)
    t_train = time.time() - t1
    ch = sel.choose(Xte)
    r_mlp = selector.regret(Tte, ch)
    r_model = selector.regret(Tte, selector.analytic_choices(te, cands, selector.default_model_params(sms)))
    fitted, train_regret = selector.fit_model_params(tr, Ttr, cands, sms)
    r_fit = selector.regret(Tte, selector.analytic_choices(te, cands, fitted))
    # a fixed default: last-block, full grid (8 CTAs/SM), 16-byte vectors
    fixed = [i for i, c in enumerate(cands) if c.variant == sr.LAST_BLOCK and c.grid == 8 * sms and
             c.vec_bytes == 16][0]
    r_fixed = selector.regret(Tte, np.full(len(te), fixed))
    # inference cost of one shape: device time per call of the predict kernel
    # in a CUDA graph of 200 calls, and per eager call (host launch included)
    x1 = torch.from_numpy(((Xte[:1] - sel.mu) / sel.sd).astype(np.float32)).cuda()
    cls = torch.empty(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    infer_us = _graph_time(torch, torch.cuda.Stream(), lambda: sel.mlp.predict(x1, cls), 200) * 1e3
    infer_eager_us = _time_calls(torch, lambda: sel.mlp.predict(x1, cls), 200, st) * 1e3
    # one whole per-call choice (features, predict, class read back) for a shape not seen before
    nat = sel.native(cands)
    t0 = time.perf_counter()
    for i in range(50):
        nat.choose((1 << 20) + 4096 * i, sr.F32)
    choose_us = (time.perf_counter() - t0) / 50 * 1e6
    nat.close()

    def summ(r):
        return {"mean": round(float(r.mean()), 4), "median": round(float(np.median(r)), 4),
                "p90": round(float(np.quantile(r, 0.9)), 4), "max": round(float(r.max()), 4),
                "within_5pct": round(float(np.mean(r <= 0.05)), 4)}
    _emit({"suite": "selector", "train_shapes": len(tr), "train_timings": int(np.isfinite(Ttr).sum()),
           "heldout_shapes": len(te), "candidates": len(cands), "collect_s": round(t_collect, 1),
           "train_s": round(t_train, 1), "final_loss": losses[-1][1], "regret_mlp": summ(r_mlp),
           "regret_model": summ(r_model), "regret_model_fitted": summ(r_fit),
           "model_fitted_params": {f: round(getattr(fitted, f), 3) for f in selector.FIT_FIELDS},
           "regret_fixed_default": summ(r_fixed),
           "mlp_inference_us_per_call": round(infer_us, 2), "mlp_inference_eager_us_per_call": round(infer_eager_us, 2),
           "first_choice_us_per_shape": round(choose_us, 2)})
    return 0


def barrier_suite(args):
    import torch
    import paper_2004_05371_gb300 as sr
    sr.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    def run(level, **kw):
        try:
            r = sr.barrier_bench(level, **kw)
            _emit({"suite": "barrier", "level": level, **kw, **{k: (round(v, 3) if isinstance(v, float) else v)
                                                                for k, v in r.items()}})
        except sr.SRError as e:
            _emit({"suite": "barrier", "level": level, **kw, "error": str(e)})
    iters = 100_000      # back-to-back syncs per measurement (r1; the differential's r2 = r1 / 10)

    def block_counts(threads):
        """1, 2, 4, ... up to one CTA per SM, the SM count itself, then whole
        waves of 2, 4, 8, ... CTAs per SM up to what is resident at once."""
        out = [b for b in (1, 2, 4, 8, 16, 32, 64, 128) if b < sms] + [sms]
        k = 2
        while k * threads <= 2048 and k <= 32:
            out.append(k * sms)
            k *= 2
        return out
    for g in (1, 2, 4, 8, 16, 32):
        run(sr.LEVEL_WARP, group=g, iters=iters)
    for blocks in block_counts(1024):
        run(sr.LEVEL_WARP, group=32, blocks=blocks, threads=1024, iters=iters)
    for g in (1, 2, 7, 16, 31, 32):
        run(sr.LEVEL_COALESCED, group=g, iters=iters)
    run(sr.LEVEL_SHUFFLE, iters=iters)
    for t in (32, 128, 256, 1024):                     # Section V-B: block sync against active warps
        for blocks in block_counts(t):
            run(sr.LEVEL_BLOCK, blocks=blocks, threads=t, iters=iters)
    for c in (2, 4, 8, 16):
        for t in (128, 1024):
            for blocks in sorted({c, 8 * c, c * (sms // c)}):
                run(sr.LEVEL_CLUSTER, cluster=c, threads=t, blocks=blocks, iters=iters)
    for t in (32, 128, 256, 512, 1024):                # Section V-C: grid sync over blocks/SM x threads/block
        for blocks in block_counts(t):
            run(sr.LEVEL_GRID, blocks=blocks, threads=t, iters=iters)
    for kind in (sr.LAUNCH_TRADITIONAL, sr.LAUNCH_COOPERATIVE, sr.LAUNCH_CLUSTER):   # Table I
        run(sr.LEVEL_KERNEL, reps=20, method=kind)
    run(sr.LEVEL_KERNEL, reps=20, method=sr.LAUNCH_COOPERATIVE, blocks=sms)
    run(sr.LEVEL_KERNEL, reps=20, method=sr.LAUNCH_CLUSTER, cluster=16, blocks=16)
    run(sr.LEVEL_FADD, iters=1_000_000)
    for fp32 in (0, sr.WR_FP32):                                                     # Table V
        for m in range(7):
            run(sr.LEVEL_WARP_REDUCE, method=m | fp32, iters=20000)
            run(sr.LEVEL_WARP_REDUCE, method=m | fp32, iters=20000, threads=1024)
    return 0


def precision_suite(args):
    import torch
    import oracle
    import paper_2004_05371_gb300 as sr
    import workloads
    sr.load()
    n = 1 << 28
    st = torch.cuda.current_stream()
    cases = []
    x = workloads.lognormal_f32(n, seed=0, sigma=4.0)
    cases.append(("lognormal_s4", "f32", x, None))
    bits = workloads.to_bf16_bits(x)
    cases.append(("lognormal_s4", "bf16", bits, None))
    codes, deq = workloads.to_e4m3_codes(x)
    cases.append(("lognormal_s4", "fp8", codes, deq))
    del x
    for cond in (1e4, 1e5, 1e6, 1e7, 1e8):
        cases.append(("cancel_%.0e" % cond, "f32", workloads.cancelling_f32(n, cond=cond, seed=0), None))
    for name, dt, arr, scale in cases:
        if dt == "f32":
            exact, s64, sabs = oracle.exact_f32(arr), oracle.sum_f32(arr), oracle.sum_abs_f32(arr)
            xd = torch.from_numpy(arr).cuda()
        elif dt == "bf16":
            exact, s64 = oracle.exact_bf16(arr), oracle.sum_bf16(arr)
            dec = np.frombuffer((arr.astype(np.uint32) << 16).tobytes(), dtype=np.float32)
            sabs = oracle.sum_abs_f32(dec)
            xd = torch.from_numpy(arr.view(np.int16)).cuda().view(torch.bfloat16)
        else:
            exact, s64 = oracle.exact_e4m3(arr, scale), oracle.sum_e4m3(arr, scale)
            sabs = oracle.sum_e4m3(arr & 0x7F, scale)
            xd = torch.from_numpy(arr).cuda()
        S = oracle.to_float(exact)
        cond = sabs / abs(S) if S else float("inf")
        for mode, flags in (("plain", 0), ("kahan", sr.F_KAHAN), ("kahan+fp64", sr.F_KAHAN | sr.F_FP64_COMBINE),
                            ("kahan+fp64_auto", sr.F_FP64_AUTO)):
            cfg = sr.make_config(sr.AUTO | flags, scale=scale or 0.0)  # last-block-done at this size
            out = sr.reduce_sum(xd, config=cfg)
            got = float(out.item())
            ms = _time_calls(torch, lambda: sr.reduce_sum(xd, config=cfg, out=out), 30, st)
            _emit({"suite": "precision", "input": name, "dtype": dt, "mode": mode, "n": n,
                   "cond": cond, "exact": S, "fp64_oracle": s64, "gpu": got,
                   "abs_err": abs(got - S), "rel_err": abs(got - S) / abs(S) if S else None,
                   "err_vs_fp64_oracle": abs(got - s64), "fp64_oracle_err": abs(s64 - S),
                   "gate_plain_4eps_sumabs": 4 * 2.0 ** -23 * sabs,
                   "gate_kahan_abs": (2 * 2.0 ** -24 + n * 2.0 ** -48) * sabs,
                   "gbs": round(xd.numel() * xd.element_size() / (ms * 1e-3) / 1e9, 1)})
        del xd
        torch.cuda.empty_cache()
    return 0


def _graph_time(torch, stream, body, calls, reps=3):
    """Device time per call (ms) of `body` captured `calls` times into one
    CUDA graph on `stream`, averaged over `reps` replays after one warm replay."""
    with torch.cuda.stream(stream):
        body()                       # warm-up (allocates the stream's workspace)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(calls):
            body()
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / (reps * calls)


def shapes_suite(args):
    """The sweeps behind SR_AUTO's table: graph-timed warm (same input every
    call) and cold (each call after a 256 MiB write, the write's own time
    subtracted) device time of LDG shapes (two-kernel and last-block; block
    256/512/1024 x vector 16/32 B x unroll 1/2/4/8, resident CTAs per SM from
    occupancy) and TMA-ring shapes, per dtype, size and compensation; SR_AUTO
    and, for FP32 / int32, CUB's DeviceReduce beside them."""
    import itertools
    import torch
    import libcmp
    import paper_2004_05371_gb300 as sr
    sr.load()
    libcmp.build()
    cmp = libcmp.lib()
    libcmp.check(cmp.cmp_prepare(1 << 30), "cmp_prepare")
    big = torch.empty(1 << 30, dtype=torch.float32, device="cuda").uniform_(-1, 1)  # 4 GiB of input bytes
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    fl = _graph_time(torch, s, lambda: flush.fill_(1), 20)
    out = torch.empty((), dtype=torch.float64, device="cuda")
    K = sr.F_KAHAN
    eb = {sr.F32: 4, sr.I32: 4, sr.BF16: 2, sr.FP8E4M3: 1}
    cases = [(sr.F32, 0, k) for k in (20, 22, 24, 26, 27, 28, 30)] + [(sr.F32, K, k) for k in (26, 27, 28, 30)]
    cases += [(dt, c, k) for dt in (sr.BF16, sr.FP8E4M3) for c in (0, K) for k in (28, 30)]
    # compensated inputs of 2, 16 and 64 MiB (the two-kernel regime below 64 MiB)
    comp_mid = [(sr.F32, K, k) for k in (19, 22, 24)] + [(sr.BF16, K, k) for k in (20, 23, 25)]
    comp_mid += [(sr.FP8E4M3, K, k) for k in (21, 24, 26)]
    # plain BF16, FP8 and int32 below 512 MiB, and int32 above
    gaps = [(sr.BF16, 0, k) for k in (20, 23, 25, 26, 27)] + [(sr.FP8E4M3, 0, k) for k in (21, 24, 26, 27)]
    gaps += [(sr.I32, 0, k) for k in (19, 22, 24, 26, 28)]
    which = getattr(args, "shape_cases", "all")
    cases = {"comp_mid": comp_mid, "gaps": gaps}.get(which, cases + comp_mid + gaps)
    for dt, comp, k in cases:
        n = 1 << k
        calls = 40 if k <= 22 else (8 if k <= 26 else 3)
        cfgs = [("auto", sr.make_config(sr.AUTO | comp))]
        for st, blk, vec, un in itertools.product((sr.TWO_KERNEL, sr.LAST_BLOCK), (256, 512, 1024), (16, 32),
                                                  (1, 2, 4, 8)):
            cfgs.append(("%s %dx%dB u%d" % ("two_kernel" if st == sr.TWO_KERNEL else "last_block", blk, vec, un),
                         sr.make_config(st | comp, block_threads=blk, vec_bytes=vec, unroll=un)))
        for t, stg, blk in ((32768, 4, 160), (32768, 4, 544), (65536, 2, 288), (65536, 2, 544), (65536, 3, 544),
                            (16384, 6, 288)):
            cfgs.append(("last_block ring %dKx%d %d" % (t >> 10, stg, blk),
                         sr.make_config(sr.LAST_BLOCK | sr.F_BULK | comp, tile_bytes=t, stages=stg, block_threads=blk)))
        res = []

        def timed(name, fn):
            try:
                w = _graph_time(torch, s, fn, calls)
                c = _graph_time(torch, s, lambda: (flush.fill_(1), fn()), calls) - fl
            except Exception:
                torch.cuda.synchronize()
                return
            res.append((name, round(w * 1e3, 2), round(c * 1e3, 2)))
        for name, cfg in cfgs:
            timed(name, lambda cfg=cfg: sr.check(sr.reduce_sum_ptr(big.data_ptr(), n, dt, out.data_ptr(), cfg,
                                                                   torch.cuda.current_stream().cuda_stream)))
        if dt == sr.F32 and not comp:
            timed("cub", lambda: libcmp.check(cmp.cmp_cub_sum_f32(big.data_ptr(), n, out.data_ptr(),
                                                                   torch.cuda.current_stream().cuda_stream), "cub"))
        bw = min(r[1] for r in res)
        bc = min(r[2] for r in res)
        _emit({"suite": "shapes", "dtype": dt, "compensated": bool(comp), "log2n": k, "bytes": n * eb[dt],
               "auto": [r for r in res if r[0] == "auto"], "cub": [r for r in res if r[0] == "cub"],
               "best_warm": sorted(res, key=lambda r: r[1])[:4], "best_cold": sorted(res, key=lambda r: r[2])[:4],
               "best_both": sorted(res, key=lambda r: max(r[1] / bw, r[2] / bc))[:4]})
    return 0


def sweep_suite(args):
    """Device time per call, from CUDA graphs of back-to-back calls (no host
    launch cost): warm = the same input every call; cold = each call preceded
    by a 256 MiB buffer write (L2 flush), the flush-only graph's time
    subtracted."""
    import torch
    import paper_2004_05371_gb300 as sr
    sr.load()
    import libcmp
    libcmp.build()
    cmp = libcmp.lib()
    libcmp.check(cmp.cmp_prepare(1 << 30), "cmp_prepare")
    big = torch.empty(1 << 30, dtype=torch.float32, device="cuda").uniform_(-1, 1)
    bigi = big.view(torch.int32)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()

    def graph_time(body, calls):
        return _graph_time(torch, s, body, calls)

    fl_ms = graph_time(lambda: flush.fill_(1), 20)
    for dt, src in (("f32", big), ("i32", bigi)):
        for k in range(10, 31):
            n = 1 << k
            x = src[:n]
            calls = 200 if k <= 20 else (20 if k <= 26 else 4)
            for name, v in (("auto", sr.AUTO), ("two_kernel", sr.TWO_KERNEL), ("atomic", sr.ATOMIC),
                            ("last_block", sr.LAST_BLOCK), ("grid_sync", sr.GRID_SYNC),
                            ("single_cluster_8", sr.SINGLE_CLUSTER | sr.CLUSTER(3)),
                            ("single_cta", sr.SINGLE_CLUSTER), ("last_block_cluster4", sr.LAST_BLOCK | sr.CLUSTER(2)),
                            ("last_block_bulk", sr.LAST_BLOCK | sr.F_BULK)):
                if name in ("single_cluster_8", "single_cta") and k > 24:
                    continue
                cfg = sr.make_config(v)
                out = torch.empty((), dtype=torch.int64 if dt == "i32" else torch.float32, device="cuda")

                def call():
                    sr.check(sr.reduce_sum_ptr(x.data_ptr(), n, sr.I32 if dt == "i32" else sr.F32, out.data_ptr(),
                                               cfg, torch.cuda.current_stream().cuda_stream))
                try:
                    warm = graph_time(call, calls)
                    both = graph_time(lambda: (flush.fill_(1), call()), max(4, calls // 10))
                except Exception as e:  # e.g. a launch form that stream capture does not accept
                    _emit({"suite": "sweep", "dtype": dt, "log2n": k, "variant": name, "error": str(e)[:160]})
                    torch.cuda.synchronize()
                    continue
                cold = max(both - fl_ms, 1e-6)
                _emit({"suite": "sweep", "dtype": dt, "log2n": k, "variant": name,
                       "warm_us": round(warm * 1e3, 2), "cold_us": round(cold * 1e3, 2),
                       "warm_gbs": round(n * 4 / (warm * 1e-3) / 1e9, 1),
                       "cold_gbs": round(n * 4 / (cold * 1e-3) / 1e9, 1)})
            # library reference point (not on the path): CUB's DeviceReduce, warm and cold
            cub_out = torch.empty((), dtype=torch.int64 if dt == "i32" else torch.float32, device="cuda")
            cub_fn = cmp.cmp_cub_sum_i32 if dt == "i32" else cmp.cmp_cub_sum_f32

            def cub_call():
                libcmp.check(cub_fn(x.data_ptr(), n, cub_out.data_ptr(), torch.cuda.current_stream().cuda_stream),
                             "cub")
            warm = graph_time(cub_call, calls)
            both = graph_time(lambda: (flush.fill_(1), cub_call()), max(4, calls // 10))
            cold = max(both - fl_ms, 1e-6)
            _emit({"suite": "sweep", "dtype": dt, "log2n": k, "variant": "cub DeviceReduce (library reference)",
                   "warm_us": round(warm * 1e3, 2), "cold_us": round(cold * 1e3, 2),
                   "warm_gbs": round(n * 4 / (warm * 1e-3) / 1e9, 1),
                   "cold_gbs": round(n * 4 / (cold * 1e-3) / 1e9, 1)})
            # library reference point (not on the path): PyTorch's own reduction kernel
            if dt == "f32":
                try:
                    warm = graph_time(lambda: torch.sum(x), calls)
                    _emit({"suite": "sweep", "dtype": dt, "log2n": k, "variant": "torch.sum (library reference)",
                           "warm_us": round(warm * 1e3, 2), "warm_gbs": round(n * 4 / (warm * 1e-3) / 1e9, 1)})
                except Exception as e:
                    _emit({"suite": "sweep", "dtype": dt, "log2n": k, "variant": "torch.sum", "error": str(e)[:120]})
    return 0


def segmented_suite(args):
    """The batched workload alone: 10,000 lognormal segments (median 4096,
    sigma 1.94, clipped to [1, 2^24]) totalling about args.n FP32 elements,
    in one library-owned graph launch per step (also the ncu capture target)."""
    import torch
    import paper_2004_05371_gb300 as sr
    import workloads
    sr.load()
    nseg = 10_000
    off = workloads.segment_offsets(nseg, args.n, seed=0)
    n = int(off[-1])
    x = torch.from_numpy(workloads.uniform_f32(n, seed=0)).cuda()
    od = torch.from_numpy(off).cuda()
    out = torch.empty(nseg, dtype=torch.float32, device="cuda")
    if args.variant is not None:
        cfg = sr.make_config(args.variant)
    else:  # tile / vector width / grid / stage from the exhaustive autotuner
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        cands = sr.candidates(sms, full=True)
        us = sr.autotune(x.data_ptr(), n, sr.F32, out.data_ptr(), cands, reps=3, offsets_ptr=od.data_ptr(),
                         nseg=nseg)
        cfg = cands[int(np.argmin(us))]
    sr.check(sr.reduce_sum_segmented_ptr(x.data_ptr(), od.data_ptr(), nseg, sr.F32, out.data_ptr(), cfg))
    g = sr.SegmentedGraph(x, od, out, cfg)
    st = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        g.launch(st)
    ms = _time_calls(torch, lambda: g.launch(st), args.steps, st)
    r = sr.plan_segmented(nseg, sr.F32, cfg)
    _emit({"suite": "segmented", "n": n, "nseg": nseg, "us_per_launch": round(ms * 1e3, 2),
           "gbs": round(n * 4 / (ms * 1e-3) / 1e9, 1), "stage": r.variant & sr.STAGE_MASK, "grid": r.grid,
           "block": r.block_threads, "vec_bytes": r.vec_bytes, "unroll": r.unroll})
    g.close()
    return 0


def seglayouts_suite(args):
    """The segmented kernel across layouts at ~2^28 FP32 elements: 10,000 and
    100,000 lognormal segments, 1M / 4M / 16M equal ones (268, 64 and 16
    elements), 4M lognormal short ones (median 40, empty ones included); the
    default kernel and SR_F_DENSE_SEGMENTS in two launch shapes, the TMA
    form (SR_F_BULK, 256 threads, chunks of 4 rows, 2 stages) and the
    warp-per-segment form (SR_F_WARP_SEGMENTS, 16 B x 4 and 16 B x 2) and the
    thread-per-segment form (SR_F_LANE_SEGMENTS, 4 loads per step) and the
    adaptive form (SR_F_ADAPTIVE_SEGMENTS); atomic finish where a form has one;
    device time per call in a CUDA graph."""
    import torch
    import paper_2004_05371_gb300 as sr
    import workloads
    sr.load()
    N = 1 << 28
    NX = N + (1 << 22)  # lognormal totals land within 1 % of N: the buffer covers offsets[nseg]
    x = torch.empty(NX, dtype=torch.float32, device="cuda").uniform_(-1, 1)
    s = torch.cuda.Stream()
    cases = [("10k lognormal (median 4096)", workloads.segment_offsets(10_000, N, seed=0)),
             ("100k lognormal (median 2684)", workloads.segment_offsets(100_000, N, seed=0, median=N // 100_000)),
             ("1M equal (268)", np.linspace(0, N, 1_000_001).astype(np.int64)),
             ("4M equal (64)", np.arange(4_194_305, dtype=np.int64) * 64),
             ("16M equal (16)", np.arange(16_777_217, dtype=np.int64) * 16),
             ("4M lognormal (median 40, empties)",
              workloads.segment_offsets(4 << 20, N, seed=3, median=40, sigma=1.5, lo=0, hi=1 << 16))]
    forms = {"ldg256": ((256, 32, 8), 0), "dense256": ((256, 32, 8), sr.F_DENSE_SEGMENTS),
             "ldg512": ((512, 32, 4), 0), "dense512": ((512, 32, 4), sr.F_DENSE_SEGMENTS),
             "tma": ((256, 32, 4), sr.F_BULK), "warp16": ((256, 16, 4), sr.F_WARP_SEGMENTS),
             "warp16u2": ((256, 16, 2), sr.F_WARP_SEGMENTS), "lane": ((256, 16, 4), sr.F_LANE_SEGMENTS),
             "lane32": ((256, 32, 4), sr.F_LANE_SEGMENTS), "adaptive": ((256, 16, 2), sr.F_ADAPTIVE_SEGMENTS)}
    only = getattr(args, "layout", None)
    form = getattr(args, "seg_form", None)
    chosen = set(form.split(",")) if form else None
    if chosen and not chosen <= set(forms):
        raise SystemExit("unknown --seg-form: %s" % ",".join(sorted(chosen - set(forms))))
    for name, off in cases:
        if only and only not in name:
            continue
        nseg, n = len(off) - 1, int(off[-1])
        if n > NX:
            raise RuntimeError("layout %s needs %d elements, buffer holds %d" % (name, n, NX))
        od = torch.from_numpy(off).cuda()
        out = torch.empty(nseg, dtype=torch.float32, device="cuda")
        for key, (shape, flags) in forms.items():
            if chosen and key not in chosen:
                continue
            cfg = sr.make_config(sr.ATOMIC | flags, block_threads=shape[0], vec_bytes=shape[1], unroll=shape[2],
                                 stages=2 if flags & sr.F_BULK else 0)

            def call(cfg=cfg):
                sr.check(sr.reduce_sum_segmented_ptr(x.data_ptr(), od.data_ptr(), nseg, sr.F32, out.data_ptr(),
                                                     cfg, torch.cuda.current_stream().cuda_stream))
            ms = _graph_time(torch, s, call, 5, reps=4)
            r = sr.plan_segmented(nseg, sr.F32, cfg)  # the shape that ran (dense lowers unroll 8 to 4)
            _emit({"suite": "seglayouts", "layout": name, "nseg": nseg, "n": n,
                   "dense": bool(flags & sr.F_DENSE_SEGMENTS), "bulk": bool(flags & sr.F_BULK),
                   "warp": bool(flags & sr.F_WARP_SEGMENTS), "lane": bool(flags & sr.F_LANE_SEGMENTS),
                   "adaptive": bool(flags & sr.F_ADAPTIVE_SEGMENTS),
                   "form": key, "shape": "%d threads x %d B x unroll %d" % shape,
                   "ran": "%d threads x %d B x unroll %d%s" % (r.block_threads, r.vec_bytes, r.unroll,
                                                               ", %d stages" % r.stages if r.stages else ""),
                   "us": round(ms * 1e3, 2),
                   "gbs": round(n * 4 / (ms * 1e-3) / 1e9, 1)})
        del od, out
        torch.cuda.empty_cache()
    return 0


def latency_suite(args):
    """Small-n latency: device time per call of single-cluster shapes (no grid
    stage; 1-16 CTAs of 128-512 threads, 16/32-byte vectors, unroll 1/2/4) in
    CUDA graphs of 400 calls at n = 2^10..2^18 FP32, the five fastest per
    size and SR_AUTO beside them; then a direct A/B of four cluster shapes
    (graphs of 1000 calls, median of 5 alternating repetitions) at 2^14..2^18."""
    import torch
    import paper_2004_05371_gb300 as sr
    import workloads
    sr.load()
    s = torch.cuda.Stream()
    out = torch.empty((), dtype=torch.float32, device="cuda")

    def per_call_us(x, n, cfg, calls, reps):
        def body():
            sr.check(sr.reduce_sum_ptr(x.data_ptr(), n, sr.F32, out.data_ptr(), cfg,
                                       torch.cuda.current_stream().cuda_stream))
        return _graph_time(torch, s, body, calls, reps=reps) * 1e3

    for k in (10, 12, 14, 16, 18):
        n = 1 << k
        x = torch.from_numpy(workloads.uniform_f32(n, seed=0)).cuda()
        timed = []
        for lc in range(5):
            for blk in (128, 256, 512):
                for vec in (16, 32):
                    for un in (1, 2, 4):
                        cfg = sr.make_config(sr.SINGLE_CLUSTER | sr.CLUSTER(lc), block_threads=blk, vec_bytes=vec,
                                             unroll=un)
                        try:
                            sr.plan(n, sr.F32, cfg)
                            timed.append((per_call_us(x, n, cfg, 400, 5), 1 << lc, blk, vec, un))
                        except sr.SRError:
                            continue  # shape not launchable at this size
        timed.sort()
        for us, ctas, blk, vec, un in timed[:5]:
            _emit({"suite": "latency", "log2n": k, "shape": "%d CTA x %d threads, %d B x %d" % (ctas, blk, vec, un),
                   "us_per_call": round(us, 3)})
        _emit({"suite": "latency", "log2n": k, "shape": "SR_AUTO",
               "us_per_call": round(per_call_us(x, n, sr.make_config(sr.AUTO), 400, 5), 3)})
    shapes = {"8 x 128": (3, 128), "16 x 256": (4, 256), "8 x 256": (3, 256), "16 x 128": (4, 128)}
    for k in (14, 16, 17, 18):
        n = 1 << k
        x = torch.from_numpy(workloads.uniform_f32(n, seed=0)).cuda()
        res = {name: [] for name in shapes}
        for _ in range(5):
            for name, (lc, blk) in shapes.items():
                cfg = sr.make_config(sr.SINGLE_CLUSTER | sr.CLUSTER(lc), block_threads=blk, vec_bytes=32, unroll=2)
                res[name].append(per_call_us(x, n, cfg, 1000, 5))
        _emit({"suite": "latency_ab", "log2n": k,
               **{name: round(sorted(v)[2], 3) for name, v in res.items()},
               "spread": {name: round(max(v) - min(v), 3) for name, v in res.items()}})
    return 0


def run(name, args):
    return {"selector": selector_suite, "barrier": barrier_suite, "precision": precision_suite, "shapes": shapes_suite,
            "sweep": sweep_suite, "segmented": segmented_suite, "seglayouts": seglayouts_suite,
            "latency": latency_suite}[name](args)
