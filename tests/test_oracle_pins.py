"""Pins for the CPU oracle against facts that do not come from the oracle itself:
closed forms, exact rational arithmetic (fractions.Fraction), Shewchuk's
correctly rounded math.fsum, PyTorch's CPU FP8/BF16 casts, and the values the
paper prints in Tables III and IV.  No GPU needed."""
import json
import math
import os
import random
import struct
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from oracle import model
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ int32 / int64
@pytest.mark.parametrize("n", [0, 1, 2, 3, 1000, 65535, 65536, 65537, (1 << 20) + 3])
def test_int_closed_form_sum_1_to_n(n):
    x = np.arange(1, n + 1, dtype=np.int32)
    assert oracle.sum_i32(x) == n * (n + 1) // 2


def test_int_worst_case_extremes():
    n = 1 << 22
    assert oracle.sum_i32(np.full(n, 2**31 - 1, np.int32)) == n * (2**31 - 1)
    assert oracle.sum_i32(np.full(n, -(2**31), np.int32)) == -n * 2**31


def test_int_brute_force_python_ints():
    rng = random.Random(7)
    for n in [0, 1, 31, 32, 33, 1023, 1025]:
        vals = [rng.randint(-(2**31), 2**31 - 1) for _ in range(n)]
        assert oracle.sum_i32(np.array(vals, np.int32)) == sum(vals)


def test_int_permutation_invariance():
    x = workloads.uniform_i32(100_003, seed=0)
    p = np.random.default_rng(1).permutation(x.size)
    assert oracle.sum_i32(x) == oracle.sum_i32(x[p])


# ------------------------------------------------------- FP64 loop, floats
@pytest.mark.parametrize("n", [1, 2, 4095, 4096])
def test_fp_closed_form_integer_valued(n):
    x = np.arange(1, n + 1, dtype=np.float32)
    assert oracle.sum_f32(x) == n * (n + 1) / 2
    assert oracle.to_float(oracle.exact_f32(x)) == n * (n + 1) / 2


def test_fp_constant_and_alternating():
    n = 1 << 20
    assert oracle.sum_f32(np.ones(n, np.float32)) == n
    alt = np.tile(np.array([1.0, -1.0], np.float32), n // 2)
    assert oracle.sum_f32(alt) == 0.0
    assert oracle.sum_f32(np.append(alt, np.float32(1.0))) == 1.0
    c = np.float32(2.0 ** -5)
    altc = np.tile(np.array([c, -c], np.float32), 1000)
    assert oracle.exact_f32(altc) == 0
    assert oracle.exact_f32(np.append(altc, c)) == Fraction(1, 32)


def test_fp_constant_tenth_closed_form():
    n = 1 << 20
    x = np.full(n, 0.1, np.float32)
    fl = Fraction(float(np.float32(0.1)))
    assert oracle.exact_f32(x) == n * fl


def _fraction_sum(vals):
    return sum((Fraction(float(v)) for v in vals), Fraction(0))


def test_exact_vs_fraction_bruteforce_specials():
    tiny = struct.unpack("<f", struct.pack("<I", 1))[0]          # 2^-149
    fmax = float(np.finfo(np.float32).max)
    sub = struct.unpack("<f", struct.pack("<I", 0x007FFFFF))[0]  # largest subnormal
    cases = [
        [], [tiny], [tiny, -tiny], [fmax, fmax, fmax, fmax], [fmax, -fmax, tiny],
        [sub, tiny, -1.5, 2.0 ** 100, -(2.0 ** 100)], [-0.0, 0.0, -0.0],
    ]
    rng = np.random.default_rng(3)
    for n in [1, 2, 3, 31, 32, 33, 127, 128, 129]:
        cases.append(list(rng.uniform(-1, 1, n).astype(np.float32)))
        cases.append(list((rng.standard_normal(n) * 2.0 ** rng.integers(-140, 120, n)).astype(np.float32)))
    for vals in cases:
        x = np.array(vals, dtype=np.float32)
        assert oracle.exact_f32(x) == _fraction_sum(x), vals


@pytest.mark.parametrize("gen", ["uniform", "lognormal", "cancel"])
def test_exact_rounding_equals_fsum(gen):
    """Both are correctly rounded to binary64, so they must agree bit for bit."""
    n = 200_000
    if gen == "uniform":
        x = workloads.uniform_f32(n, seed=0)
    elif gen == "lognormal":
        x = workloads.lognormal_f32(n, seed=0, sigma=4.0)
    else:
        x = workloads.cancelling_f32(n, cond=1e8, seed=0)
    ref = math.fsum(x.astype(np.float64).tolist())
    assert oracle.to_float(oracle.exact_f32(x)) == ref


def test_fp64_loop_within_its_own_bound():
    x = workloads.lognormal_f32(300_000, seed=2, sigma=4.0)
    exact = oracle.exact_f32(x)
    s64 = oracle.sum_f32(x)
    sabs = math.fsum(np.abs(x.astype(np.float64)).tolist())
    bound = (x.size - 1) * 2.0 ** -53 * sabs * (1 + 1e-12)
    assert abs(Fraction(s64) - exact) <= Fraction(bound)


def test_sum_abs():
    x = workloads.uniform_f32(10_001, seed=4)
    assert oracle.sum_abs_f32(x) == pytest.approx(math.fsum(np.abs(x.astype(np.float64))), rel=1e-12)


# ------------------------------------------------------------ decoding
def test_e4m3_decode_all_codes_vs_torch():
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    for c in range(256):
        v = oracle.decode_e4m3(c)
        if math.isnan(ref[c]):
            assert math.isnan(v), c
        else:
            assert v == ref[c], (c, v, ref[c])
    assert oracle.decode_e4m3(0x7E) == 448.0
    assert oracle.decode_e4m3(0x01) == 2.0 ** -9
    assert oracle.decode_e4m3(0x38) == 1.0


def test_bf16_decode_vs_torch():
    bits = np.arange(0, 65536, 7, dtype=np.uint16)
    ref = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    for b, r in zip(bits.tolist(), ref.tolist()):
        v = oracle.decode_bf16(b)
        assert (math.isnan(v) and math.isnan(r)) or v == r, (b, v, r)


def test_bf16_sums_vs_fsum():
    x = workloads.lognormal_f32(50_000, seed=5, sigma=4.0)
    bits = workloads.to_bf16_bits(x)
    dec = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    assert oracle.to_float(oracle.exact_bf16(bits)) == math.fsum(dec.tolist())
    assert oracle.sum_bf16(bits) == pytest.approx(math.fsum(dec.tolist()), rel=1e-9, abs=1e-300)


def test_e4m3_sums_vs_fraction():
    x = workloads.lognormal_f32(4000, seed=6, sigma=2.0)
    codes, deq = workloads.to_e4m3_codes(x)
    dec = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    exact = sum((Fraction(float(d)) for d in dec), Fraction(0)) * Fraction(deq)
    assert oracle.exact_e4m3(codes, deq) == exact
    assert oracle.sum_e4m3(codes, deq) == pytest.approx(float(exact), rel=1e-12)


# ------------------------------------------------------------ segmented
def test_segmented_closed_forms_and_empty():
    lens = [0, 1, 2, 0, 100, 4096, 0, 3]
    off = np.zeros(len(lens) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    x = np.concatenate([np.arange(1, L + 1) for L in lens]).astype(np.int32) if sum(lens) else np.zeros(0, np.int32)
    got = oracle.segsum_i32(x, off)
    assert got.tolist() == [L * (L + 1) // 2 for L in lens]
    gotf = oracle.segsum_f32(x.astype(np.float32), off)
    assert gotf.tolist() == [L * (L + 1) / 2 for L in lens]
    assert oracle.segexact_f32(x.astype(np.float32), off).tolist() == [L * (L + 1) / 2 for L in lens]


def test_segmented_partition_of_total():
    off = workloads.random_segment_offsets(500, 300, seed=3)
    x = workloads.uniform_i32(int(off[-1]), seed=3)
    seg = oracle.segsum_i32(x, off)
    assert int(seg.sum()) == oracle.sum_i32(x)
    xf = workloads.uniform_f32(int(off[-1]), seed=3)
    ex = oracle.segexact_f32(xf, off)
    for s in [0, 17, 250, 499]:
        a, b = off[s], off[s + 1]
        assert ex[s] == math.fsum(xf[a:b].astype(np.float64).tolist())


# ---------------------------------------------------- performance model
def _tables():
    with open(os.path.join(GOLDEN, "perf_model_tables.json")) as f:
        return json.load(f)


def test_table_III_concurrency_is_littles_law():
    g = _tables()
    tol = g["tolerance_rel"]
    for gpu, row in g["table_III"].items():
        T = row["latency_cycles"]
        for cfg, bw in row["bw_B_per_cycle"].items():
            printed = row["concurrency_B"][cfg]
            assert model.concurrency(T, bw) == pytest.approx(printed, rel=tol), (gpu, cfg)


def test_table_IV_switch_points():
    g = _tables()
    tol = g["tolerance_rel"]
    for gpu, rows in g["table_IV"].items():
        T = g["table_III"][gpu]["latency_cycles"]
        bw = g["table_III"][gpu]["bw_B_per_cycle"]
        for name, r in rows.items():
            tb, tm = bw[r["basic"]], bw[r["more"]]
            assert model.switch_point_l(r["t_sync"], tb, tm) == pytest.approx(r["N_l"], rel=tol), (gpu, name)
            assert model.switch_point_m(T, r["t_sync"], tb) == pytest.approx(r["N_m"], rel=tol), (gpu, name)


@pytest.mark.parametrize("T,ts,tb,tm", [(13.0, 110.0, 0.62, 19.6), (13.0, 420.0, 19.6, 215.0),
                                        (18.5, 2135.0, 13.8, 141.0), (50.0, 5.0, 10.0, 100.0),
                                        (800.0, 2000.0, 30.0, 7000.0)])
def test_eq2_decision_matches_closed_switch_point(T, ts, tb, tm):
    """Eqs. 4 and 5 are the solutions of Eq. 2 in their scenarios: scanning N,
    Eq. 2 must flip exactly at switch_point()."""
    sp = model.switch_point(T, ts, tb, tm)
    for N in np.geomspace(0.5, 50 * max(sp, 1.0), 4000):
        if abs(N - sp) <= 1e-9 * sp:
            continue
        assert model.prefer_basic(N, T, ts, tb, tm) == (N < sp), (N, sp)


def test_eq6_recovers_planted_overhead():
    O, w = 1081.0, 1000.0           # ns per launch, ns per wait unit
    for i, j in [(5, 1), (10, 2), (7, 3)]:
        lat_ij = i * O + i * j * w
        lat_ji = j * O + j * i * w
        assert model.launch_overhead(lat_ij, lat_ji, i, j) == pytest.approx(O, rel=1e-12)


def test_eq7_eq8_against_simulation():
    rng = np.random.default_rng(11)
    t_true, base, r1, r2 = 3.7, 5000.0, 100_000, 1_000
    s1, s2 = 40.0, 25.0
    N = 20_000
    L1 = base + r1 * t_true + rng.normal(0, s1, N)
    L2 = base + r2 * t_true + rng.normal(0, s2, N)
    t, sigma = model.differential_latency(L1.tolist(), L2.tolist(), r1, r2)
    assert t == pytest.approx(t_true, rel=1e-3)
    d = (L1 - L2) / (r1 - r2)
    assert sigma == pytest.approx(float(np.std(d, ddof=1)), rel=0.03)
    assert sigma == pytest.approx(math.hypot(s1, s2) / (r1 - r2), rel=0.03)


# ------------------------------------------------------- error bounds
def test_gamma_and_stated_bound():
    assert oracle.gamma(1) == pytest.approx(2.0 ** -24 / (1 - 2.0 ** -24))
    assert oracle.stated_fp32_bound(1.0) == 4 * 2.0 ** -23
    # recursive FP32 summation of 1 + tiny*k: the error is within gamma_{n-1} sum|x|
    x = np.full(4097, np.float32(2.0 ** -24))
    x[0] = 1.0
    acc = np.float32(0)
    for v in x:
        acc = np.float32(acc + v)
    err = abs(Fraction(float(acc)) - oracle.exact_f32(x))
    assert err <= Fraction(oracle.fp32_tree_bound(float(np.sum(np.abs(x), dtype=np.float64)), x.size - 1))


# ------------------------------------------------------------- MLP oracle
def test_mlp_oracle_closed_forms():
    from oracle import mlp
    dims = (3, 5, 4)
    zero = np.zeros(mlp.param_count(dims))
    X = np.random.default_rng(0).normal(size=(7, 3))
    Q = np.eye(4)[[0, 1, 2, 3, 0, 1, 2]]
    # all-zero network: uniform softmax, loss log K, d/db3 = mean(1/K - q)
    assert mlp.loss(zero, X, Q, dims) == pytest.approx(math.log(4))
    g = mlp.grad(zero, X, Q, dims)
    assert np.allclose(g[-4:], (0.25 - Q).mean(axis=0))
    assert np.allclose(g[:-4], 0.0)
    # 1-1-2 network by hand: z = (ab c, ab d) for x = 1, a, b > 0
    a, b, c, d = 0.7, 1.3, 0.4, -0.9
    p = np.array([a, 0.0, b, 0.0, c, d, 0.0, 0.0])
    z0, z1 = a * b * c, a * b * d
    assert mlp.loss(p, [[1.0]], [[1.0, 0.0]], (1, 1, 2)) == pytest.approx(math.log1p(math.exp(z1 - z0)))


def test_mlp_oracle_gradient_vs_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(1)
    dims = (6, 8, 5)
    p = rng.normal(scale=0.5, size=mlp.param_count(dims))
    X = rng.normal(size=(9, 6))
    Q = rng.dirichlet(np.ones(5), size=9)
    g = mlp.grad(p, X, Q, dims)
    h = 1e-6
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss(p + e, X, Q, dims) - mlp.loss(p - e, X, Q, dims)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), k


def test_mlp_oracle_adam_first_step_is_sign_step():
    from oracle import mlp
    g = np.array([0.3, -2.0, 1e-3])
    p1, m, v = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    # bias-corrected first step: mhat = g, vhat = g^2, so the step is lr * sign(g)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-4)


def test_mlp_oracle_predict_and_forward_by_hand():
    """The 1-1-2 network worked by hand: x = 1 gives z = (abc + 0.1, abd + 0.2),
    class 0 for c > d; x = -1 is cut by the first ReLU, so z = b3 and the
    class is argmax(b3) = 1."""
    from oracle import mlp
    a, b, c, d = 0.7, 1.3, 0.4, -0.9
    p = np.array([a, 0.0, b, 0.0, c, d, 0.1, 0.2])
    _, _, z = mlp.forward(p, [[1.0], [-1.0]], (1, 1, 2))
    assert z[0] == pytest.approx([a * b * c + 0.1, a * b * d + 0.2])
    assert z[1] == pytest.approx([0.1, 0.2])
    assert list(mlp.predict(p, [[1.0], [-1.0]], (1, 1, 2))) == [0, 1]


def test_segsum_abs_closed_form():
    x = np.array([1, -2, 3, -4, 5, -6], np.float32)
    off = np.array([0, 2, 2, 6], np.int64)
    assert list(oracle.segsum_abs_f32(x, off)) == [3.0, 0.0, 18.0]
