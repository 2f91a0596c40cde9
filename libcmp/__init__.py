"""CUB's DeviceReduce as a library comparison point for the benchmark
suites (not part of the library; never on its path).  build() compiles
libcmp/cub_sum.cu for sm_103a into libcmp/libcub_sum.so."""
import ctypes
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cub_sum.cu")
LIB = os.path.join(HERE, "libcub_sum.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                                                            os.path.getmtime(__file__)):
        return LIB
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-shared", SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (SRC, r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError("libcub_sum.so is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.cmp_prepare.argtypes = [i64]
        L.cmp_prepare.restype = ctypes.c_int
        for f in (L.cmp_cub_sum_f32, L.cmp_cub_sum_i32):
            f.argtypes = [vp, i64, vp, vp]
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def check(err: int, what: str):
    if err != 0:
        raise RuntimeError("%s failed: cudaError %d" % (what, err))
