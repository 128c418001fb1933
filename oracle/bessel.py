"""Bessel-Chebyshev coefficients of the time-evolution operator (FP64).

App. B (Eq. cheb_relation and the coefficient equation below it) gives the
Jacobi-Anger expansion
    exp(-i H~ tau~) = sum_n c_n(tau~) T_n(H~),  c_0 = J_0(tau~),  c_n = 2 (-i)^n J_n(tau~).
J_n(x) for n = 0..n_max is computed with Miller's backward recurrence
    J_{k-1}(x) = (2k/x) J_k(x) - J_{k+1}(x)
started far above both n_max and x and normalised with J_0 + 2 sum_k J_{2k} = 1
(J. C. P. Miller, British Association Mathematical Tables, vol. X, 1952;
Abramowitz & Stegun 9.1.27 and 9.1.46).

Truncation (Sec. II.A): the paper keeps the terms with |c_n| > eta, eta = 1e-14.  Read
literally ("for all n < N") the rule would stop at the first small coefficient below
tau~; the reading used here is N(tau~) = 1 + max{n : |c_n(tau~)| > eta}, so the sum
runs over n = 0..N-1.  This reading reproduces the paper's expansion load R(pi) ~ 6
and the 1/2, 1/3, 1/4, 1/5 ratios of Fig. 2(b).

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import functools
import math

import numpy as np

ETA = 1e-14


def miller_start(n_max: int, x: float) -> int:
    m = int(max(n_max, math.ceil(abs(x)))) + 60 + int(12.0 * abs(x) ** (1.0 / 3.0))
    return m + (m & 1)  # even, so the normalisation sum ends on J_0


def bessel_j_sequence(x: float, n_max: int) -> np.ndarray:
    """J_0(x) .. J_{n_max}(x) in FP64 by Miller's backward recurrence."""
    out = np.zeros(n_max + 1)
    if x == 0.0:
        out[0] = 1.0
        return out
    ax = abs(float(x))
    m = miller_start(n_max, ax)
    vals = np.zeros(m + 2)
    vals[m + 1] = 0.0
    vals[m] = 1e-300
    norm = 0.0
    for k in range(m, 0, -1):
        vals[k - 1] = (2.0 * k / ax) * vals[k] - vals[k + 1]
        if abs(vals[k - 1]) > 1e200:       # rescale to stay in range
            vals[k - 1:] *= 1e-200
            norm *= 1e-200
        if (k - 1) % 2 == 0 and k - 1 > 0:
            norm += 2.0 * vals[k - 1]
    norm += vals[0]
    out[:] = vals[: n_max + 1] / norm
    if x < 0:                                # J_n(-x) = (-1)^n J_n(x)
        out[1::2] *= -1.0
    return out


def cheb_coefficients(tau: float, n_terms: int) -> np.ndarray:
    """c_n(tau~) for n = 0..n_terms-1 (complex128)."""
    J = bessel_j_sequence(tau, max(n_terms - 1, 0))
    n = np.arange(n_terms)
    phase = (-1j) ** (n % 4)
    c = 2.0 * phase * J[:n_terms]
    c[0] = J[0]
    return c.astype(np.complex128)


def _scan_limit(tau: float) -> int:
    return int(math.ceil(abs(tau) + 40.0 + 12.0 * abs(tau) ** (1.0 / 3.0)))


@functools.lru_cache(maxsize=65536)
def truncation_order(tau: float, eta: float = ETA) -> int:
    """N(tau~) = 1 + max{n : |c_n(tau~)| > eta}."""
    n_scan = _scan_limit(tau)
    c = np.abs(cheb_coefficients(tau, n_scan + 1))
    big = np.flatnonzero(c > eta)
    if big.size == 0:
        return 1
    if big[-1] >= n_scan - 5:
        raise RuntimeError("coefficient scan too short")
    return int(big[-1]) + 1


def expansion_load(tau: float, eta: float = ETA) -> float:
    """R(tau~) = N(tau~) / tau~ (Sec. II.A, Fig. 2)."""
    return truncation_order(tau, eta) / tau
