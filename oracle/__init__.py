"""CPU oracle for the device-wide sum reduction — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and its ``--impl reference`` arm) may import this
package.  The product path (``paper_2004_05371_gb300``) never imports it;
the two share no code.

The operator is the paper's case study (Section VII, "Case Study:
Reduction Operator"): summing the elements of an array.  The oracle is
that definition, S = sum_i x_i, as sequential loops in ``sr_oracle.c``
(int64 for int32 input, FP64 and an exact fixed-point accumulator for
floating point), wrapped here with ctypes.  ``model.py`` holds the paper's
performance model (Eqs. 1-5) and its measurement formulas (Eqs. 6-8).

Pins (tests/test_oracle_pins.py): closed forms (sum 1..n), integer-valued
floating-point arrays, exact comparison with ``math.fsum`` (Shewchuk,
correctly rounded) and ``fractions.Fraction`` brute force, FP8/BF16 decode
against PyTorch's CPU casts, Table III / Table IV values for the model.
"""
import ctypes
from fractions import Fraction

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, f64, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        L.oracle_limbs.restype = ctypes.c_int
        L.oracle_sum_i32.restype = i64
        L.oracle_sum_i32.argtypes = [vp, i64]
        for name in ("oracle_sum_f32", "oracle_sum_bf16", "oracle_sum_abs_f32"):
            getattr(L, name).restype = f64
            getattr(L, name).argtypes = [vp, i64]
        L.oracle_sum_e4m3.restype = f64
        L.oracle_sum_e4m3.argtypes = [vp, i64, f64]
        for name in ("oracle_exact_f32", "oracle_exact_bf16", "oracle_exact_e4m3"):
            getattr(L, name).restype = ctypes.c_int
            getattr(L, name).argtypes = [vp, i64, vp]
        L.oracle_decode_e4m3.restype = f64
        L.oracle_decode_e4m3.argtypes = [ctypes.c_uint8]
        L.oracle_decode_bf16.restype = f64
        L.oracle_decode_bf16.argtypes = [ctypes.c_uint16]
        L.oracle_segsum_f32.restype = None
        L.oracle_segsum_f32.argtypes = [vp, vp, i64, vp]
        L.oracle_segsum_abs_f32.restype = None
        L.oracle_segsum_abs_f32.argtypes = [vp, vp, i64, vp]
        L.oracle_segsum_i32.restype = None
        L.oracle_segsum_i32.argtypes = [vp, vp, i64, vp]
        L.oracle_segexact_f32.restype = ctypes.c_int
        L.oracle_segexact_f32.argtypes = [vp, vp, i64, vp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    a = np.ascontiguousarray(a)
    assert a.dtype == dtype, (a.dtype, dtype)
    return a


# ------------------------------------------------------------ plain sums
def sum_i32(x) -> int:
    """Exact sum of int32 values in int64 (sequential loop)."""
    x = _c(x, np.int32)
    return int(lib().oracle_sum_i32(_ptr(x), x.size))


def sum_f32(x) -> float:
    """Sequential FP64 sum of binary32 values."""
    x = _c(x, np.float32)
    return float(lib().oracle_sum_f32(_ptr(x), x.size))


def sum_abs_f32(x) -> float:
    x = _c(x, np.float32)
    return float(lib().oracle_sum_abs_f32(_ptr(x), x.size))


def sum_bf16(bits) -> float:
    """Sequential FP64 sum of BF16 values given as their uint16 bit patterns."""
    bits = _c(bits, np.uint16)
    return float(lib().oracle_sum_bf16(_ptr(bits), bits.size))


def sum_e4m3(codes, scale: float) -> float:
    """Sequential FP64 sum of scale * decode(code) over FP8 E4M3 codes."""
    codes = _c(codes, np.uint8)
    return float(lib().oracle_sum_e4m3(_ptr(codes), codes.size, float(scale)))


# ------------------------------------------------------------ exact sums
def _limbs_to_int(L) -> int:
    v = 0
    for k, d in enumerate(L):
        v += int(d) << (32 * k)
    return v


def _exact(fn, arr) -> Fraction:
    L = np.zeros(lib().oracle_limbs(), dtype=np.int64)
    rc = fn(_ptr(arr), arr.size, _ptr(L))
    if rc != 0:
        raise ValueError("non-finite input")
    return Fraction(_limbs_to_int(L), 1 << 149)


def exact_f32(x) -> Fraction:
    """Exact rational value of sum(x) for binary32 x (fixed-point accumulator)."""
    return _exact(lib().oracle_exact_f32, _c(x, np.float32))


def exact_bf16(bits) -> Fraction:
    return _exact(lib().oracle_exact_bf16, _c(bits, np.uint16))


def exact_e4m3(codes, scale) -> Fraction:
    """Exact value of scale * sum(decode(codes)) (scale taken as its exact
    binary value)."""
    return _exact(lib().oracle_exact_e4m3, _c(codes, np.uint8)) * Fraction(float(scale))


def to_float(q: Fraction) -> float:
    """Correctly rounded conversion (int / int true division rounds once)."""
    return q.numerator / q.denominator


def decode_e4m3(code: int) -> float:
    return float(lib().oracle_decode_e4m3(int(code)))


def decode_bf16(bits: int) -> float:
    return float(lib().oracle_decode_bf16(int(bits)))


# ------------------------------------------------------------- segmented
def segsum_f32(x, offsets):
    x = _c(x, np.float32)
    offsets = _c(offsets, np.int64)
    out = np.zeros(offsets.size - 1, dtype=np.float64)
    lib().oracle_segsum_f32(_ptr(x), _ptr(offsets), out.size, _ptr(out))
    return out


def segsum_abs_f32(x, offsets):
    x = _c(x, np.float32)
    offsets = _c(offsets, np.int64)
    out = np.zeros(offsets.size - 1, dtype=np.float64)
    lib().oracle_segsum_abs_f32(_ptr(x), _ptr(offsets), out.size, _ptr(out))
    return out


def segsum_i32(x, offsets):
    x = _c(x, np.int32)
    offsets = _c(offsets, np.int64)
    out = np.zeros(offsets.size - 1, dtype=np.int64)
    lib().oracle_segsum_i32(_ptr(x), _ptr(offsets), out.size, _ptr(out))
    return out


def segexact_f32(x, offsets):
    """Per-segment exact sums as a float64 array of correctly rounded values."""
    x = _c(x, np.float32)
    offsets = _c(offsets, np.int64)
    nseg = offsets.size - 1
    NL = lib().oracle_limbs()
    L = np.zeros(nseg * NL, dtype=np.int64)
    if lib().oracle_segexact_f32(_ptr(x), _ptr(offsets), nseg, _ptr(L)) != 0:
        raise ValueError("non-finite input")
    L = L.reshape(nseg, NL)
    return np.array([to_float(Fraction(_limbs_to_int(row), 1 << 149)) for row in L])


# --------------------------------------------------------- error bounds
U32 = 2.0 ** -24          # binary32 unit roundoff
EPS32 = 2.0 ** -23        # FLT_EPSILON


def gamma(m: int, u: float = U32) -> float:
    """Higham's gamma_m = m u / (1 - m u): the relative bound of m rounded
    operations in a chain (Accuracy and Stability of Numerical Algorithms,
    Lemma 3.1)."""
    mu = m * u
    assert mu < 1.0
    return mu / (1.0 - mu)


def fp32_tree_bound(sum_abs: float, chain: int) -> float:
    """Absolute bound gamma_chain * sum|x| for any summation whose longest
    path from a leaf to the root has `chain` FP32 additions."""
    return gamma(chain) * sum_abs


def stated_fp32_bound(sum_abs: float) -> float:
    """The plain FP32 tree gate: |S_gpu - S_exact| <= 4 * eps32 * sum|x_i|."""
    return 4.0 * EPS32 * sum_abs
