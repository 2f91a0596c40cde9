"""Python binding of ``libsr.so`` (the C ABI declared in ``include/sr.h``).

Argument marshalling only: every step of the reduction runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams; no torch kernel is
used on the path.  If the library has not been built this module raises: there
is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsr.so")

# dtypes (sr_dtype)
F32, I32, BF16, FP8E4M3 = 0, 1, 2, 3
# grid stages (sr_stage)
AUTO, TWO_KERNEL, ATOMIC, LAST_BLOCK, GRID_SYNC, SINGLE_CLUSTER = 0, 1, 2, 3, 4, 5
STAGE_NAMES = {AUTO: "auto", TWO_KERNEL: "two_kernel", ATOMIC: "atomic", LAST_BLOCK: "last_block",
               GRID_SYNC: "grid_sync", SINGLE_CLUSTER: "single_cluster"}
STAGE_MASK = 0xF
CLUSTER_SHIFT = 4
CLUSTER_MASK = 0x70
F_KAHAN = 0x100
F_FP64_COMBINE = 0x200
F_BULK = 0x400
F_HOST_DIRECT = 0x800
F_FP64_AUTO = 0x1000
F_DENSE_SEGMENTS = 0x2000
F_WARP_SEGMENTS = 0x4000  # segmented: whole segments per warp, no grid stage
F_LANE_SEGMENTS = 0x8000  # segmented: whole segments per thread, no grid stage
F_ADAPTIVE_SEGMENTS = 0x10000  # segmented: one cooperative launch, partition by length on the device
# status codes (sr_status)
OK, ERR_ARG, ERR_DTYPE, ERR_LAUNCH, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
# barrier levels (sr_level)
(LEVEL_WARP, LEVEL_COALESCED, LEVEL_BLOCK, LEVEL_CLUSTER, LEVEL_GRID, LEVEL_KERNEL, LEVEL_SHUFFLE, LEVEL_FADD,
 LEVEL_WARP_REDUCE) = range(9)
# sr_warp_reduce_method (Table V) and sr_launch_kind (Table I)
(WR_SERIAL, WR_NOSYNC, WR_VOLATILE_TILE, WR_TILE, WR_COALESCED, WR_TILE_SHUFFLE,
 WR_COALESCED_SHUFFLE) = range(7)
WR_FP32 = 16
LAUNCH_TRADITIONAL, LAUNCH_COOPERATIVE, LAUNCH_CLUSTER = range(3)


def CLUSTER(log2c: int) -> int:
    return (log2c & 7) << CLUSTER_SHIFT


class Config(ctypes.Structure):
    """Mirror of ``sr_config``."""
    _fields_ = [("variant", ctypes.c_int), ("block_threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("grid", ctypes.c_int), ("vec_bytes", ctypes.c_int), ("unroll", ctypes.c_int),
                ("tile_bytes", ctypes.c_int), ("stages", ctypes.c_int), ("scale", ctypes.c_float),
                ("reserved", ctypes.c_int * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BarrierConfig(ctypes.Structure):
    """Mirror of ``sr_barrier_config``."""
    _fields_ = [("level", ctypes.c_int), ("iters", ctypes.c_int64), ("blocks", ctypes.c_int),
                ("threads", ctypes.c_int), ("cluster", ctypes.c_int), ("group", ctypes.c_int),
                ("reps", ctypes.c_int), ("method", ctypes.c_int)]


class BarrierResult(ctypes.Structure):
    """Mirror of ``sr_barrier_result``."""
    _fields_ = [("cycles_per_sync", ctypes.c_double), ("ns_per_sync", ctypes.c_double),
                ("ns_sigma", ctypes.c_double), ("syncs_per_cycle_per_sm", ctypes.c_double),
                ("clock_mhz", ctypes.c_double), ("null_kernel_total_ns", ctypes.c_double),
                ("blocks", ctypes.c_int), ("threads", ctypes.c_int), ("correct", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ModelParams(ctypes.Structure):
    """Mirror of ``sr_model_params``."""
    _fields_ = [("sms", ctypes.c_int), ("hbm_bytes_per_ns", ctypes.c_double), ("mem_latency_ns", ctypes.c_double),
                ("launch_ns", ctypes.c_double), ("grid_sync_ns", ctypes.c_double),
                ("last_block_ns", ctypes.c_double), ("atomic_ns", ctypes.c_double), ("per_cta_ns", ctypes.c_double),
                ("per_segment_ns", ctypes.c_double)]


class SRError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        if status == ERR_CUDA and _lib is not None:
            msg += " (cudaError %d)" % _lib.sr_last_cuda_error()
        super().__init__("%s%s" % (what + ": " if what else "", msg))


_lib = None


def load():
    """Load the CUDA library; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsr.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.sr_reduce_sum.restype = i32
    L.sr_reduce_sum.argtypes = [vp, i64, i32, vp, i32, vp]
    L.sr_reduce_sum_segmented_checked.restype = i32
    L.sr_reduce_sum_segmented_checked.argtypes = [vp, i64, vp, i64, i32, vp, ctypes.POINTER(Config), vp]
    L.sr_reduce_sum_ex.restype = i32
    L.sr_reduce_sum_ex.argtypes = [vp, i64, i32, vp, ctypes.POINTER(Config), vp]
    L.sr_reduce_sum_noalloc.restype = i32
    L.sr_reduce_sum_noalloc.argtypes = [vp, i64, i32, vp, ctypes.POINTER(Config), vp]
    L.sr_reduce_sum_segmented.restype = i32
    L.sr_reduce_sum_segmented.argtypes = [vp, vp, i64, i32, vp, vp]
    L.sr_reduce_sum_segmented_ex.restype = i32
    L.sr_reduce_sum_segmented_ex.argtypes = [vp, vp, i64, i32, vp, ctypes.POINTER(Config), vp]
    L.sr_plan_segmented.restype = i32
    L.sr_plan_segmented.argtypes = [i64, i32, ctypes.POINTER(Config), ctypes.POINTER(Config)]
    L.sr_graph_capture_segmented.restype = i32
    L.sr_graph_capture_segmented.argtypes = [vp, vp, i64, i32, vp, ctypes.POINTER(Config), ctypes.POINTER(vp)]
    L.sr_graph_launch.restype = i32
    L.sr_graph_launch.argtypes = [vp, vp]
    L.sr_graph_destroy.restype = i32
    L.sr_graph_destroy.argtypes = [vp]
    L.sr_barrier_bench.restype = i32
    L.sr_barrier_bench.argtypes = [i32, i64]
    L.sr_barrier_bench_ex.restype = i32
    L.sr_barrier_bench_ex.argtypes = [ctypes.POINTER(BarrierConfig), ctypes.POINTER(BarrierResult)]
    L.sr_barrier_bench_last.restype = i32
    L.sr_barrier_bench_last.argtypes = [ctypes.POINTER(BarrierResult)]
    L.sr_differential_latency.restype = i32
    L.sr_differential_latency.argtypes = [vp, i64, vp, i64, i64, i64, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
    L.sr_candidates.restype = i32
    L.sr_candidates.argtypes = [i32, i32, ctypes.POINTER(Config), i32]
    L.sr_autotune.restype = i32
    L.sr_autotune.argtypes = [vp, i64, vp, i64, i32, vp, ctypes.POINTER(Config), i32, i32,
                              ctypes.POINTER(ctypes.c_float), vp]
    L.sr_select_analytic.restype = i32
    L.sr_select_analytic.argtypes = [ctypes.POINTER(ModelParams), i64, i32, i64, ctypes.POINTER(Config), i32,
                                     ctypes.POINTER(ctypes.c_float)]
    L.sr_mlp_create.restype = i32
    L.sr_mlp_create.argtypes = [i32, i32, i32, ctypes.POINTER(vp)]
    L.sr_mlp_destroy.restype = i32
    L.sr_mlp_destroy.argtypes = [vp]
    L.sr_mlp_param_count.restype = i64
    L.sr_mlp_param_count.argtypes = [vp]
    L.sr_mlp_set_params.restype = i32
    L.sr_mlp_set_params.argtypes = [vp, vp, i64]
    L.sr_mlp_get_params.restype = i32
    L.sr_mlp_get_params.argtypes = [vp, vp, i64]
    L.sr_mlp_train_step.restype = i32
    L.sr_mlp_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp, vp]
    L.sr_mlp_predict.restype = i32
    L.sr_mlp_predict.argtypes = [vp, vp, i32, vp, vp, vp]
    L.sr_selector_features.restype = i32
    L.sr_selector_features.argtypes = [i64, i32, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_float)]
    L.sr_reduce_sum_host.restype = i32
    L.sr_reduce_sum_host.argtypes = [vp, i64, i32, vp, ctypes.POINTER(Config), vp]
    L.sr_mlp_dims.restype = i32
    L.sr_mlp_dims.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.sr_selector_create.restype = i32
    L.sr_selector_create.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(Config), i32, ctypes.POINTER(vp)]
    L.sr_selector_destroy.restype = i32
    L.sr_selector_destroy.argtypes = [vp]
    L.sr_selector_choose.restype = i32
    L.sr_selector_choose.argtypes = [vp, i64, i32, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(Config), vp]
    L.sr_reduce_sum_selected.restype = i32
    L.sr_reduce_sum_selected.argtypes = [vp, vp, i64, i32, vp, vp]
    L.sr_segmented_layout_flags.restype = i32
    L.sr_segmented_layout_flags.argtypes = [i32, i32, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.sr_reduce_sum_segmented_selected.restype = i32
    L.sr_reduce_sum_segmented_selected.argtypes = [vp, vp, vp, i64, i32, vp, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_double, vp]
    L.sr_selftest_bounded_wait.restype = i32
    L.sr_selftest_bounded_wait.argtypes = [ctypes.c_uint64, vp]
    L.sr_stream_release.restype = i32
    L.sr_stream_release.argtypes = [vp]
    L.sr_stream_status.restype = i32
    L.sr_stream_status.argtypes = [vp]
    L.sr_plan.restype = i32
    L.sr_plan.argtypes = [i64, i32, ctypes.POINTER(Config), ctypes.POINTER(Config)]
    L.sr_parse_variant.restype = i32
    L.sr_parse_variant.argtypes = [ctypes.c_char_p, ctypes.POINTER(i32)]
    L.sr_tune_save.restype = i32
    L.sr_tune_save.argtypes = [ctypes.c_char_p]
    L.sr_tune_load.restype = i32
    L.sr_tune_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(i64)]
    L.sr_tune_size.restype = i64
    L.sr_tune_size.argtypes = []
    L.sr_tune_clear.restype = i32
    L.sr_tune_clear.argtypes = []
    L.sr_selector_save.restype = i32
    L.sr_selector_save.argtypes = [vp, ctypes.c_char_p]
    L.sr_selector_load.restype = i32
    L.sr_selector_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
    L.sr_status_string.restype = ctypes.c_char_p
    L.sr_status_string.argtypes = [i32]
    L.sr_last_cuda_error.restype = i32
    L.sr_version.restype = ctypes.c_char_p
    _lib = L
    return L


def lib():
    return load()


def status_string(status: int) -> str:
    return lib().sr_status_string(int(status)).decode()


def version() -> str:
    return lib().sr_version().decode()


def check(status: int, what: str = ""):
    if status != OK:
        raise SRError(status, what)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(t) -> int:
    import torch
    m = {torch.float32: F32, torch.int32: I32, torch.bfloat16: BF16, torch.uint8: FP8E4M3}
    fp8 = getattr(torch, "float8_e4m3fn", None)
    if fp8 is not None:
        m[fp8] = FP8E4M3
    if t.dtype not in m:
        raise TypeError("unsupported dtype %s" % t.dtype)
    return m[t.dtype]


def out_dtype(dtype: int, variant: int):
    import torch
    if dtype == I32:
        return torch.int64
    return torch.float64 if variant & F_FP64_COMBINE else torch.float32


def make_config(variant=AUTO, **kw) -> Config:
    c = Config()
    c.variant = int(variant)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def reduce_sum_ptr(x_ptr: int, n: int, dtype: int, out_ptr: int, config: Config = None, stream=None) -> int:
    """Raw call of sr_reduce_sum_ex; returns the status (no raise)."""
    cfg = ctypes.byref(config) if config is not None else None
    return lib().sr_reduce_sum_ex(ctypes.c_void_p(x_ptr), int(n), int(dtype), ctypes.c_void_p(out_ptr), cfg,
                                  ctypes.c_void_p(_stream(stream)))


def reduce_sum_noalloc_ptr(x_ptr: int, n: int, dtype: int, out_ptr: int, config: Config = None,
                           stream=None) -> int:
    """Raw call of sr_reduce_sum_noalloc (no device allocation); returns the status."""
    cfg = ctypes.byref(config) if config is not None else None
    return lib().sr_reduce_sum_noalloc(ctypes.c_void_p(x_ptr), int(n), int(dtype), ctypes.c_void_p(out_ptr), cfg,
                                       ctypes.c_void_p(_stream(stream)))


def reduce_sum_host_ptr(x_ptr: int, n: int, dtype: int, out_ptr: int, config: Config = None, stream=None) -> int:
    """Raw call of sr_reduce_sum_host (HOST input and output pointers)."""
    cfg = ctypes.byref(config) if config is not None else None
    return lib().sr_reduce_sum_host(ctypes.c_void_p(x_ptr), int(n), int(dtype), ctypes.c_void_p(out_ptr), cfg,
                                    ctypes.c_void_p(_stream(stream)))


def reduce_sum(x, variant: int = AUTO, out=None, config: Config = None, stream=None, **cfg_fields):
    """Sum of a contiguous 1-D CUDA tensor through sr_reduce_sum_ex.

    Returns a 0-dim CUDA tensor (int64 for int32 input, float64 with
    F_FP64_COMBINE, float32 otherwise).  uint8 input is read as FP8 E4M3 codes.
    """
    import torch
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    dt = dtype_code(x)
    if config is None:
        config = make_config(variant, **cfg_fields)
    if out is None:
        out = torch.empty((), dtype=out_dtype(dt, config.variant), device=x.device)
    st = reduce_sum_ptr(x.data_ptr(), x.numel(), dt, out.data_ptr(), config, stream)
    check(st, "sr_reduce_sum_ex")
    return out


def reduce_sum_segmented_ptr(x_ptr: int, offsets_ptr: int, nseg: int, dtype: int, out_ptr: int,
                             config: Config = None, stream=None) -> int:
    """Raw call of sr_reduce_sum_segmented_ex; returns the status (no raise)."""
    cfg = ctypes.byref(config) if config is not None else None
    return lib().sr_reduce_sum_segmented_ex(ctypes.c_void_p(x_ptr), ctypes.c_void_p(offsets_ptr), int(nseg),
                                            int(dtype), ctypes.c_void_p(out_ptr), cfg,
                                            ctypes.c_void_p(_stream(stream)))


def reduce_sum_segmented_checked_ptr(x_ptr: int, n_elems: int, offsets_ptr: int, nseg: int, dtype: int,
                                     out_ptr: int, config: Config = None, stream=None) -> int:
    """Raw call of sr_reduce_sum_segmented_checked (offsets validated on the
    device against n_elems); returns the launch status.  A failed check shows
    up as SR_ERR_ARG from stream_status()."""
    cfg = ctypes.byref(config) if config is not None else None
    return lib().sr_reduce_sum_segmented_checked(ctypes.c_void_p(x_ptr), int(n_elems), ctypes.c_void_p(offsets_ptr),
                                                 int(nseg), int(dtype), ctypes.c_void_p(out_ptr), cfg,
                                                 ctypes.c_void_p(_stream(stream)))


def reduce_sum_segmented(x, offsets, variant: int = AUTO, out=None, config: Config = None, stream=None,
                         **cfg_fields):
    """Per-segment sums of a CUDA tensor over int64 CSR offsets (CUDA tensor of
    nseg + 1 entries).  Returns a CUDA tensor of nseg results."""
    import torch
    if not (x.is_cuda and offsets.is_cuda and x.is_contiguous() and offsets.is_contiguous()):
        raise ValueError("x and offsets must be contiguous CUDA tensors")
    if offsets.dtype != torch.int64:
        raise TypeError("offsets must be int64")
    dt = dtype_code(x)
    if config is None:
        config = make_config(variant, **cfg_fields)
    nseg = offsets.numel() - 1
    if out is None:
        out = torch.empty(max(nseg, 0), dtype=out_dtype(dt, config.variant), device=x.device)
    st = reduce_sum_segmented_ptr(x.data_ptr(), offsets.data_ptr(), nseg, dt, out.data_ptr(), config, stream)
    check(st, "sr_reduce_sum_segmented_ex")
    return out


def plan_segmented(nseg: int, dtype: int, config: Config = None) -> Config:
    r = Config()
    cfg = ctypes.byref(config) if config is not None else None
    check(lib().sr_plan_segmented(int(nseg), int(dtype), cfg, ctypes.byref(r)), "sr_plan_segmented")
    return r


class SegmentedGraph:
    """A segmented sum captured once into a library-owned CUDA graph
    (sr_graph_capture_segmented); launch() replays it with one graph launch.
    The tensors must stay alive (and in place) until close()."""

    def __init__(self, x, offsets, out, config: Config = None):
        self._keep = (x, offsets, out)
        self._h = ctypes.c_void_p()
        cfg = ctypes.byref(config) if config is not None else None
        check(lib().sr_graph_capture_segmented(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(offsets.data_ptr()),
                                               offsets.numel() - 1, dtype_code(x), ctypes.c_void_p(out.data_ptr()),
                                               cfg, ctypes.byref(self._h)), "sr_graph_capture_segmented")

    def launch(self, stream=None):
        check(lib().sr_graph_launch(self._h, ctypes.c_void_p(_stream(stream))), "sr_graph_launch")

    def close(self):
        if self._h:
            lib().sr_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def barrier_bench(level: int, iters: int = 0, blocks: int = 0, threads: int = 0, cluster: int = 0,
                  group: int = 0, reps: int = 0, method: int = 0) -> dict:
    """sr_barrier_bench_ex: one barrier-latency measurement (raises on error)."""
    c = BarrierConfig(level, iters, blocks, threads, cluster, group, reps, method)
    r = BarrierResult()
    check(lib().sr_barrier_bench_ex(ctypes.byref(c), ctypes.byref(r)), "sr_barrier_bench_ex")
    return r.as_dict()


def differential_latency(L1, L2, r1: int, r2: int):
    """Eqs. 7-8 computed by the library's host code: returns (t, sigma)."""
    a = (ctypes.c_double * len(L1))(*L1)
    b = (ctypes.c_double * len(L2))(*L2)
    t, sg = ctypes.c_double(), ctypes.c_double()
    check(lib().sr_differential_latency(a, len(L1), b, len(L2), int(r1), int(r2), ctypes.byref(t),
                                        ctypes.byref(sg)), "sr_differential_latency")
    return t.value, sg.value


def candidates(sms: int, full: bool = False):
    """The candidate configurations (sr_candidates) as a ctypes array."""
    cnt = lib().sr_candidates(int(full), int(sms), None, 0)
    if cnt < 0:
        raise SRError(-cnt, "sr_candidates")
    arr = (Config * cnt)()
    got = lib().sr_candidates(int(full), int(sms), arr, cnt)
    if got != cnt:
        raise SRError(-got if got < 0 else ERR_ARG, "sr_candidates")
    return arr


def autotune(x_ptr: int, n: int, dtype: int, out_ptr: int, cands, reps: int = 5, offsets_ptr: int = 0,
             nseg: int = 0, stream=None):
    """sr_autotune: microseconds per call for every candidate (inf = cannot run)."""
    us = (ctypes.c_float * len(cands))()
    check(lib().sr_autotune(ctypes.c_void_p(x_ptr), int(n), ctypes.c_void_p(offsets_ptr or None), int(nseg),
                            int(dtype), ctypes.c_void_p(out_ptr), cands, len(cands), int(reps), us,
                            ctypes.c_void_p(_stream(stream))), "sr_autotune")
    return list(us)


def select_analytic(params: ModelParams, n: int, dtype: int, nseg: int, cands):
    """sr_select_analytic: (index of the predicted-fastest candidate, predictions in us)."""
    pred = (ctypes.c_float * len(cands))()
    i = lib().sr_select_analytic(ctypes.byref(params), int(n), int(dtype), int(nseg), cands, len(cands), pred)
    if i < 0:
        raise SRError(-i, "sr_select_analytic")
    return i, list(pred)


class MLP:
    """Handle of an sr_mlp (device-resident parameters).  Argument marshalling
    only: training and inference run in the library's kernels."""

    def __init__(self, in_dim: int, hidden: int, out_dim: int):
        self.h = ctypes.c_void_p()
        check(lib().sr_mlp_create(in_dim, hidden, out_dim, ctypes.byref(self.h)), "sr_mlp_create")
        self.dims = (in_dim, hidden, out_dim)
        self.P = int(lib().sr_mlp_param_count(self.h))

    def set_params(self, host_array):
        import numpy as np
        a = np.ascontiguousarray(host_array, dtype=np.float32)
        check(lib().sr_mlp_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size), "sr_mlp_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.P, np.float32)
        check(lib().sr_mlp_get_params(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size), "sr_mlp_get_params")
        return a

    def train_step(self, X, Q, lr: float, loss=None, grad=None, stream=None):
        """X, Q: CUDA float32 tensors [B, in] / [B, out]; loss: CUDA float32
        scalar tensor (optional); grad: CUDA float32 [P] (optional)."""
        B = X.shape[0]
        check(lib().sr_mlp_train_step(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Q.data_ptr()), B,
                                      float(lr), ctypes.c_void_p(loss.data_ptr() if loss is not None else None),
                                      ctypes.c_void_p(grad.data_ptr() if grad is not None else None),
                                      ctypes.c_void_p(_stream(stream))), "sr_mlp_train_step")

    def predict(self, X, cls, logits=None, stream=None):
        check(lib().sr_mlp_predict(self.h, ctypes.c_void_p(X.data_ptr()), X.shape[0], ctypes.c_void_p(cls.data_ptr()),
                                   ctypes.c_void_p(logits.data_ptr() if logits is not None else None),
                                   ctypes.c_void_p(_stream(stream))), "sr_mlp_predict")

    def close(self):
        if self.h:
            lib().sr_mlp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selector_features(n: int, dtype: int, nseg: int, len_mean: float, len_std: float, len_max: float):
    out = (ctypes.c_float * 9)()
    check(lib().sr_selector_features(int(n), int(dtype), int(nseg), float(len_mean), float(len_std),
                                     float(len_max), out), "sr_selector_features")
    return list(out)


class NativeSelector:
    """sr_selector: a trained MLP + normalisation + candidate table, used by
    sr_reduce_sum_selected.  Keeps the MLP alive."""

    def __init__(self, mlp, mu, sd, cands):
        self.mlp, self.cands = mlp, cands
        f = ctypes.c_float * 9
        self._mu, self._sd = f(*[float(v) for v in mu]), f(*[float(v) for v in sd])
        self.h = ctypes.c_void_p()
        check(lib().sr_selector_create(mlp.h, self._mu, self._sd, cands, len(cands), ctypes.byref(self.h)),
              "sr_selector_create")

    @classmethod
    def load(cls, path):
        """A selector from a file written by save(); it owns its own MLP."""
        self = cls.__new__(cls)
        self.mlp, self.cands = None, None
        self.h = ctypes.c_void_p()
        check(lib().sr_selector_load(os.fsencode(path), ctypes.byref(self.h)), "sr_selector_load")
        return self

    def save(self, path):
        check(lib().sr_selector_save(self.h, os.fsencode(path)), "sr_selector_save")

    def choose(self, n, dtype, nseg=1, mean=None, std=0.0, mx=None, stream=None) -> Config:
        c = Config()
        mean = float(n) if mean is None else mean
        mx = float(n) if mx is None else mx
        check(lib().sr_selector_choose(self.h, int(n), int(dtype), int(nseg), float(mean), float(std), float(mx),
                                       ctypes.byref(c), ctypes.c_void_p(_stream(stream))), "sr_selector_choose")
        return c

    def close(self):
        if self.h:
            lib().sr_selector_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def parse_variant(text: str) -> int:
    v = ctypes.c_int(0)
    check(lib().sr_parse_variant(text.encode(), ctypes.byref(v)), "sr_parse_variant(%r)" % text)
    return v.value


def tune_save(path):
    check(lib().sr_tune_save(os.fsencode(path)), "sr_tune_save")


def tune_load(path) -> int:
    k = ctypes.c_int64(0)
    check(lib().sr_tune_load(os.fsencode(path), ctypes.byref(k)), "sr_tune_load")
    return k.value


def tune_size() -> int:
    return int(lib().sr_tune_size())


def tune_clear():
    check(lib().sr_tune_clear(), "sr_tune_clear")


def reduce_sum_selected_ptr(selector, x_ptr, n, dtype, out_ptr, stream=None) -> int:
    h = selector.h if selector is not None else None
    return lib().sr_reduce_sum_selected(h, ctypes.c_void_p(x_ptr), int(n), int(dtype), ctypes.c_void_p(out_ptr),
                                        ctypes.c_void_p(_stream(stream)))


def reduce_sum_segmented_selected_ptr(selector, x_ptr, offsets_ptr, nseg, dtype, out_ptr, mean, std, mx,
                                      stream=None) -> int:
    h = selector.h if selector is not None else None
    return lib().sr_reduce_sum_segmented_selected(h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(offsets_ptr),
                                                  int(nseg), int(dtype), ctypes.c_void_p(out_ptr), float(mean),
                                                  float(std), float(mx), ctypes.c_void_p(_stream(stream)))


def segmented_layout_flags(sms, dtype, nseg, mean, std, mx) -> int:
    """The form the selected segmented path applies for these statistics
    (F_DENSE_SEGMENTS, F_WARP_SEGMENTS or 0); raises on bad arguments."""
    r = lib().sr_segmented_layout_flags(int(sms), int(dtype), int(nseg), float(mean), float(std), float(mx))
    if r < 0:
        check(-r, "sr_segmented_layout_flags")
    return r


def plan(n: int, dtype: int, config: Config = None) -> Config:
    r = Config()
    cfg = ctypes.byref(config) if config is not None else None
    check(lib().sr_plan(int(n), int(dtype), cfg, ctypes.byref(r)), "sr_plan")
    return r


def stream_status(stream=None) -> int:
    return lib().sr_stream_status(ctypes.c_void_p(_stream(stream)))


def selftest_bounded_wait(limit_ns: int, stream=None) -> int:
    return lib().sr_selftest_bounded_wait(int(limit_ns), ctypes.c_void_p(_stream(stream)))


def stream_release(stream=None) -> int:
    return lib().sr_stream_release(ctypes.c_void_p(_stream(stream)))
