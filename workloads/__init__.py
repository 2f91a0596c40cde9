"""Seeded synthetic inputs shared by the tests, the bench and smoke().

This module only draws and encodes inputs; it holds none of the reduction's
arithmetic (no sums, no decoding).  Both the CUDA path and the CPU oracle
receive the arrays it returns.

Recipes (numpy ``default_rng(seed)``, PCG64):
  uniform_f32      U[-1, 1] drawn in float64, rounded to binary32.
  uniform_i32      integers uniform in [lo, hi] inclusive.
  lognormal_f32    magnitudes exp(N(mu, sigma^2)) with independent random signs.
  to_bf16_bits     binary32 -> BF16 round-to-nearest-even (PyTorch CPU cast),
                   returned as uint16 bit patterns.
  to_e4m3_codes    binary32 * scale, clamped to +-448, cast to FP8 E4M3 (OCP
                   E4M3FN, round-to-nearest-even, PyTorch CPU cast); returns
                   the uint8 codes and the dequantisation factor 1/scale.
  cancelling_f32   n/2 pairs (a_j, b_j) with b_j = -a_j - delta*|a_j| rounded
                   to binary32, shuffled; every residual a_j + b_j has the
                   same sign, so cond = sum|x| / |sum x| is about 2/delta.
                   delta is 2/cond above 2^-20; below that only a fraction
                   2^21/cond of the pairs is perturbed (by 2^-20) and the
                   rest cancel exactly (binary32 cannot carry a smaller
                   relative perturbation).  The achieved cond is measured by
                   the oracle, not assumed.
  selector_shapes  random call shapes for the selector: log2 n ~ U[10, 30],
                   dtype uniform over {f32, i32, bf16, fp8}, nseg log-uniform
                   in [1, 1e5] (at most n), segment-length sigma ~ U[0.5, 2.5].
  shape_offsets    CSR offsets of one such shape: lognormal(0, sigma) weights
                   scaled to total n (rounded; the remainder goes to the last).
  segment_offsets  CSR offsets of nseg segments whose lengths are
                   round(lognormal(ln median, sigma)) clipped to [lo, hi],
                   then scaled proportionally (and re-clipped) so that the
                   total lands within 1 % of the requested total.
"""
import numpy as np


def uniform_f32(n: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, int(n)).astype(np.float32)


def uniform_i32(n: int, seed: int = 0, lo: int = -1000, hi: int = 1000) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, int(n), endpoint=True, dtype=np.int32)


def lognormal_f32(n: int, seed: int = 0, mu: float = 0.0, sigma: float = 4.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    mag = rng.lognormal(mu, sigma, int(n))
    sign = rng.integers(0, 2, int(n)) * 2 - 1
    x = (mag * sign).astype(np.float32)
    # lognormal(0, 4) can exceed the binary32 range in principle; keep finite
    big = np.float32(3.0e38)
    return np.clip(x, -big, big)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16).copy()


def to_e4m3_codes(x: np.ndarray, scale: float = None):
    """Returns (codes uint8, dequant) with x ~= dequant * decode(codes)."""
    import torch
    x = np.ascontiguousarray(x, dtype=np.float32)
    if scale is None:
        amax = float(np.max(np.abs(x))) if x.size else 1.0
        scale = 448.0 / amax if amax > 0 else 1.0
    scale = float(np.float32(scale))
    y = np.clip(x.astype(np.float64) * scale, -448.0, 448.0).astype(np.float32)
    t = torch.from_numpy(y).to(torch.float8_e4m3fn)
    codes = t.view(torch.uint8).numpy().copy()
    dequant = float(np.float32(1.0 / scale))
    return codes, dequant


def cancelling_f32(n: int, cond: float, seed: int = 0, sigma: float = 4.0) -> np.ndarray:
    assert n % 2 == 0
    rng = np.random.default_rng(seed)
    m = n // 2
    mag = rng.lognormal(0.0, sigma, m)
    mag = np.clip(mag, 1e-30, 1e30)
    sign = rng.integers(0, 2, m) * 2 - 1
    a = (mag * sign).astype(np.float32)
    delta = 2.0 / cond
    frac = 1.0
    if delta < 2.0 ** -20:
        frac = (2.0 ** 21) / cond
        delta = 2.0 ** -20
    perturb = rng.random(m) < frac
    a64 = a.astype(np.float64)
    b = (-a64 - np.where(perturb, delta, 0.0) * np.abs(a64)).astype(np.float32)
    x = np.empty(n, dtype=np.float32)
    x[0::2] = a
    x[1::2] = b
    return x[rng.permutation(n)]


def segment_offsets(nseg: int, total: int, seed: int = 0, median: float = 4096.0,
                    sigma: float = 1.94, lo: int = 1, hi: int = 1 << 24) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lens = np.rint(rng.lognormal(np.log(median), sigma, int(nseg)))
    lens = np.clip(lens, lo, hi)
    for _ in range(20):
        s = lens.sum()
        if abs(s - total) <= 0.01 * total:
            break
        lens = np.clip(np.rint(lens * (total / s)), lo, hi)
    lens = lens.astype(np.int64)
    off = np.zeros(int(nseg) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


def random_segment_offsets(nseg: int, max_len: int, seed: int = 0,
                           p_empty: float = 0.1) -> np.ndarray:
    """Small irregular CSR layouts for parity tests: lengths uniform in
    [0, max_len] with an extra share of empty segments."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len, int(nseg), endpoint=True)
    lens[rng.random(int(nseg)) < p_empty] = 0
    off = np.zeros(int(nseg) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


def selector_shapes(count: int, seed: int):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(int(count)):
        n = int(2 ** rng.uniform(10, 30))
        nseg = int(min(n, round(10 ** rng.uniform(0, 5))))
        out.append({"n": n, "dtype": int(rng.integers(0, 4)), "nseg": max(1, nseg),
                    "sigma": float(rng.uniform(0.5, 2.5))})
    return out


def shape_offsets(shape, seed: int) -> np.ndarray:
    n, nseg = shape["n"], shape["nseg"]
    rng = np.random.default_rng(seed)
    w = rng.lognormal(0.0, shape["sigma"], nseg)
    lens = np.floor(w / w.sum() * n).astype(np.int64)
    lens[-1] += n - int(lens.sum())
    off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off
