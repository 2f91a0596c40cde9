"""The paper's performance model and measurement formulas, written out plainly.

Test infrastructure only (see ``oracle/__init__.py``).

Section VII-A ("Performance Model"):
  Eq. 1  C = T * Thr                          (Little's law: concurrency)
  Eq. 2  prefer "basic" when
         T_basic + max(0, N - C_basic)/Thr_basic < T_more + max(0, N - C_more)/Thr_more
  Eq. 3  T_more = T_basic + T_sync = T + T_sync
  Eq. 4  N_m < (T + T_sync) * Thr_basic          (C_basic < N <= C_more)
  Eq. 5  N_l < T_sync * Thr_more * Thr_basic / (Thr_more - Thr_basic)   (N > C_more)
The text takes T_basic as the latency in Little's law for BOTH concurrencies
(C_basic = T * Thr_basic, C_more = T * Thr_more); that reading is what makes
Eqs. 4 and 5 the solutions of Eq. 2 in their scenarios.

Section IX-B ("Micro-benchmark for Implicit Barriers"):
  Eq. 6  O = (Latency_ij - Latency_ji) / (i - j)
         Latency_ij: i launches, each kernel made of j wait units (and
         Latency_ji the converse), so both runs do the same i*j units of work
         and differ by (i - j) launches.
Section IX-D ("Micro-benchmark for Inter SM Instructions"):
  Eq. 7  T_instruction = (L_k1 - L_k2) / (r1 - r2)
  Eq. 8  sigma = sqrt(sigma_k1^2 + sigma_k2^2) / |r1 - r2|
         with L_ki the kernel total latency of kernel i (mean over N runs)
         and r_i its repeat count; sigma_ki the sample standard deviation.
"""
import math


# ---------------------------------------------------------------- Eq. 1
def concurrency(latency: float, throughput: float) -> float:
    return latency * throughput


# ---------------------------------------------------------------- Eq. 3
def t_more(t_basic: float, t_sync: float) -> float:
    return t_basic + t_sync


# ---------------------------------------------------------------- Eq. 2
def cost_basic(N, T, thr_basic):
    c_basic = concurrency(T, thr_basic)
    return T + max(0.0, N - c_basic) / thr_basic


def cost_more(N, T, t_sync, thr_basic, thr_more):
    c_more = concurrency(T, thr_more)
    return t_more(T, t_sync) + max(0.0, N - c_more) / thr_more


def prefer_basic(N, T, t_sync, thr_basic, thr_more) -> bool:
    """Eq. 2: True when the configuration with fewer workers is faster."""
    return cost_basic(N, T, thr_basic) < cost_more(N, T, t_sync, thr_basic, thr_more)


# ------------------------------------------------------------ Eqs. 4, 5
def switch_point_m(T, t_sync, thr_basic) -> float:
    """Eq. 4 (scenario 2, C_basic < N <= C_more)."""
    return (T + t_sync) * thr_basic


def switch_point_l(t_sync, thr_basic, thr_more) -> float:
    """Eq. 5 (scenario 3, N > C_more)."""
    return t_sync * thr_more * thr_basic / (thr_more - thr_basic)


def switch_point(T, t_sync, thr_basic, thr_more) -> float:
    """The input size below which "basic" wins, combining the three scenarios
    listed after Eq. 3: at or below C_basic basic always wins; between the
    concurrencies Eq. 4 decides; above C_more Eq. 5 decides."""
    c_basic = concurrency(T, thr_basic)
    c_more = concurrency(T, thr_more)
    n_m = switch_point_m(T, t_sync, thr_basic)
    if n_m <= c_more:
        return max(c_basic, n_m)
    return max(c_more, switch_point_l(t_sync, thr_basic, thr_more))


# ---------------------------------------------------------------- Eq. 6
def launch_overhead(latency_ij: float, latency_ji: float, i: int, j: int) -> float:
    return (latency_ij - latency_ji) / (i - j)


# ------------------------------------------------------------ Eqs. 7, 8
def _mean(v):
    return sum(v) / len(v)


def _sample_sd(v):
    m = _mean(v)
    return math.sqrt(sum((a - m) ** 2 for a in v) / (len(v) - 1))


def differential_latency(L_k1, L_k2, r1: int, r2: int):
    """Eq. 7 on the means of two independent sets of runs, and Eq. 8 for
    its standard deviation.  Returns (T_instruction, sigma)."""
    t = (_mean(L_k1) - _mean(L_k2)) / (r1 - r2)
    sigma = math.sqrt(_sample_sd(L_k1) ** 2 + _sample_sd(L_k2) ** 2) / abs(r1 - r2)
    return t, sigma
