"""Learned launch-configuration selector (no counterpart in the paper).

Orchestration only — the timings come from the library's autotuner
(sr_autotune), the features from sr_selector_features, the network is
trained by the library's MLP kernels (sr_mlp_train_step) and served by its
inference kernel (sr_mlp_predict); the baseline "method without it" is the
library's performance-model selector (sr_select_analytic, Section VII-A).

A class of the network is one of the 40 candidates of sr_candidates():
grid stage x grid size x vector width.  Targets are soft: for a shape with
per-candidate times t_c, q_c is proportional to exp(-(t_c / t_min - 1) / tau),
so candidates within a few percent of the best share the probability mass.
Regret of a choice c = t_c / t_min - 1 against the exhaustive autotuner.
"""
import ctypes
import math

import numpy as np

from . import (F32, I32, BF16, FP8E4M3, MLP, ModelParams, autotune, candidates, check, lib,
               selector_features, select_analytic)

ELEM = {F32: 4, I32: 4, BF16: 2, FP8E4M3: 1}
NFEAT = 9


def shape_stats(shape, off):
    """(mean, std, max) of the segment lengths of one shape."""
    if shape["nseg"] == 1 or off is None:
        n = float(shape["n"])
        return n, 0.0, n
    lens = np.diff(off).astype(np.float64)
    return float(lens.mean()), float(lens.std()), float(lens.max())


def features(shapes, offsets):
    X = np.zeros((len(shapes), NFEAT), np.float32)
    for i, (s, off) in enumerate(zip(shapes, offsets)):
        m, sd, mx = shape_stats(s, off)
        X[i] = selector_features(s["n"], s["dtype"], s["nseg"], m, sd, mx)
    return X


def collect_timings(shapes, offsets, cands, reps=3, device="cuda"):
    """Exhaustive autotuner timings [shapes x candidates] in microseconds."""
    import torch
    max_bytes = max(s["n"] * ELEM[s["dtype"]] for s in shapes)
    buf = torch.rand((max_bytes + 255) // 4 + 64, dtype=torch.float32, device=device)  # input bytes
    out = torch.empty(max(s["nseg"] for s in shapes) + 1, dtype=torch.float64, device=device)
    T = np.zeros((len(shapes), len(cands)), np.float64)
    for i, (s, off) in enumerate(zip(shapes, offsets)):
        if s["nseg"] > 1:
            od = torch.from_numpy(off).to(device)
            us = autotune(buf.data_ptr(), s["n"], s["dtype"], out.data_ptr(), cands, reps=reps,
                          offsets_ptr=od.data_ptr(), nseg=s["nseg"])
        else:
            us = autotune(buf.data_ptr(), s["n"], s["dtype"], out.data_ptr(), cands, reps=reps)
        T[i] = us
    torch.cuda.synchronize()
    return T


def soft_targets(T, tau=0.03):
    best = np.min(T, axis=1, keepdims=True)
    e = np.where(np.isfinite(T), np.exp(-(T / best - 1.0) / tau), 0.0)
    return (e / e.sum(axis=1, keepdims=True)).astype(np.float32)


def regret(T, choice):
    best = np.min(T, axis=1)
    return T[np.arange(len(choice)), choice] / best - 1.0


class Selector:
    """A trained network plus its feature normalisation."""

    def __init__(self, mlp, mu, sd):
        self.mlp, self.mu, self.sd = mlp, mu, sd

    def native(self, cands):
        """The C-ABI selector (sr_selector) for per-call choices."""
        from . import NativeSelector
        return NativeSelector(self.mlp, self.mu, self.sd, cands)

    def choose(self, X, device="cuda"):
        import torch
        Xn = torch.from_numpy(((X - self.mu) / self.sd).astype(np.float32)).to(device)
        cls = torch.empty(X.shape[0], dtype=torch.int32, device=device)
        self.mlp.predict(Xn, cls)
        torch.cuda.synchronize()
        return cls.cpu().numpy().astype(np.int64)


def train(X, Q, hidden=64, steps=3000, batch=256, lr=3e-3, seed=0, device="cuda", log=None):
    """Adam on the mean soft cross-entropy, minibatches from a per-epoch
    host-side permutation uploaded once per epoch (no device-side gathering)."""
    import torch
    rng = np.random.default_rng(seed)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd[sd < 1e-6] = 1.0
    Xn = ((X - mu) / sd).astype(np.float32)
    n_in, n_out = X.shape[1], Q.shape[1]
    mlp = MLP(n_in, hidden, n_out)
    # He-normal initialisation for the ReLU layers, zero biases
    p = np.concatenate([rng.normal(0, math.sqrt(2.0 / n_in), n_in * hidden), np.zeros(hidden),
                        rng.normal(0, math.sqrt(2.0 / hidden), hidden * hidden), np.zeros(hidden),
                        rng.normal(0, math.sqrt(1.0 / hidden), hidden * n_out), np.zeros(n_out)])
    mlp.set_params(p.astype(np.float32))
    loss = torch.zeros((), dtype=torch.float32, device=device)
    N = X.shape[0]
    batch = min(batch, N)
    per_epoch = N // batch
    step = 0
    losses = []
    while step < steps:
        perm = rng.permutation(N)
        Xd = torch.from_numpy(Xn[perm]).to(device)
        Qd = torch.from_numpy(Q[perm]).to(device)
        for k in range(per_epoch):
            if step >= steps:
                break
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / steps))  # cosine decay
            mlp.train_step(Xd[k * batch:(k + 1) * batch], Qd[k * batch:(k + 1) * batch], lr_t, loss=loss)
            if step % 200 == 0 or step == steps - 1:
                losses.append((step, float(loss.item())))
                if log:
                    log(step, losses[-1][1])
            step += 1
    return Selector(mlp, mu, sd), losses


def default_model_params(sms):
    """Performance-model parameters for a GB300.  HBM throughput: the
    single-array reduction at 2^28 elements.  The finishing costs are measured
    as the extra device time of each grid stage over a one-CTA call at 2^10
    elements in a CUDA graph of back-to-back calls (programmatic dependent
    launch on): a second kernel ~1.0 us (launch_ns, also the base launch),
    the atomic finish with its output-zeroing kernel ~0.7 us, last-block-done
    (fence, ticket, final reduction) ~1.5 us, a cooperative launch with
    grid.sync ~1.8 us.  Memory latency and the per-CTA and per-segment terms
    are hand-set starting values (see fit_model_params)."""
    return ModelParams(sms=sms, hbm_bytes_per_ns=6900.0, mem_latency_ns=900.0, launch_ns=1000.0,
                       grid_sync_ns=1800.0, last_block_ns=1500.0, atomic_ns=700.0, per_cta_ns=4.0,
                       per_segment_ns=150.0)


def analytic_choices(shapes, cands, params):
    return np.array([select_analytic(params, s["n"], s["dtype"], s["nseg"], cands)[0] for s in shapes],
                    dtype=np.int64)


FIT_FIELDS = ("hbm_bytes_per_ns", "mem_latency_ns", "launch_ns", "grid_sync_ns", "last_block_ns", "atomic_ns",
              "per_cta_ns", "per_segment_ns")


def fit_model_params(shapes, T, cands, sms, rounds=4, seed=0):
    """Calibrate the performance model on training timings: coordinate
    descent over log-scaled multipliers of each parameter, minimising the
    mean regret of the model's choices on the training shapes.  Gives the
    method without the network its best shot before the comparison."""
    p = default_model_params(sms)

    def score(params):
        ch = analytic_choices(shapes, cands, params)
        return float(np.mean(regret(T, ch)))

    best = score(p)
    factors = (0.25, 0.5, 0.8, 1.25, 2.0, 4.0)
    for _ in range(rounds):
        improved = False
        for f in FIT_FIELDS:
            base = getattr(p, f)
            for m in factors:
                setattr(p, f, base * m)
                sc = score(p)
                if sc < best - 1e-6:
                    best, base, improved = sc, base * m, True
            setattr(p, f, base)
        if not improved:
            break
    return p, best
