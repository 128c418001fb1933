"""Operation-count model and block-size choice, written from Sec. II.B and Tab. I (App. A).

Tab. I counts, for a fixed total duration t_tot = N_t tau with N_b = N_t / b blocks:
  DOS-Sequential      amxsy t~_tot R(tau~) = N_t N(tau~),  axpy N_t N(tau~),  dot N_t,  4 states
  DOS-Concurrent-M    amxsy t~_tot R(t~_tot)/2 = N(t~_tot)/2,  dot N(t~_tot),  3 states
  state-based block   amxsy N_b N(t~_b),  axpy N_b sum_{j=1}^{b} N(t~_j)
(one propagated direction; QE/EC/OC/DP/CD multiply by their number of propagated states).
Cost (Sec. II.B):  C(b) = N_amxsy(b) t_amxsy + N_axpy(b) t_axpy + C_other,
b_opt = argmin_b C(b).  Overall speedup from Amdahl's law (Eq. amdahl):
S = 1 / (1 - P + P/n).

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import math

from .bessel import truncation_order


def dos_sequential_counts(n_steps: int, tau: float = math.pi) -> dict:
    N = truncation_order(tau)
    return {"amxsy": n_steps * N, "axpy": n_steps * N, "dot": n_steps, "states": 4}


def dos_concurrent_m_counts(n_steps: int, tau: float = math.pi) -> dict:
    Ntot = truncation_order(n_steps * tau)
    return {"amxsy": Ntot / 2, "axpy": 0, "dot": Ntot, "states": 3}


def block_counts(n_steps: int, b: int, tau: float = math.pi) -> dict:
    """Counts of the state-based implementation with blocks of b steps (the last block may be
    shorter when b does not divide N_t)."""
    amxsy = axpy = 0
    start = 0
    while start < n_steps:
        bb = min(b, n_steps - start)
        Ns = [truncation_order(j * tau) for j in range(1, bb + 1)]
        amxsy += max(Ns)
        axpy += sum(Ns)
        start += bb
    return {"amxsy": amxsy, "axpy": axpy, "dot": n_steps}


def block_cost(n_steps: int, b: int, t_amxsy: float, t_axpy: float, tau: float = math.pi) -> float:
    c = block_counts(n_steps, b, tau)
    return c["amxsy"] * t_amxsy + c["axpy"] * t_axpy


def b_opt(n_steps: int, t_amxsy: float, t_axpy: float, b_max: int | None = None,
          tau: float = math.pi) -> int:
    b_max = n_steps if b_max is None else min(b_max, n_steps)
    best, best_c = 1, None
    for b in range(1, b_max + 1):
        c = block_cost(n_steps, b, t_amxsy, t_axpy, tau)
        if best_c is None or c < best_c:
            best, best_c = b, c
    return best


def amdahl(P: float, n: float) -> float:
    return 1.0 / (1.0 - P + P / n)
