"""Spectra from correlation values or moments (FP64), written from Sec. III.

* Fourier route (Sec. III): D(E) = (1/2pi) int exp(iEt) C(t) dt with C(-t) = C(t)*,
  sampled at t_j = j tau (tau~ = pi) and summed with the trapezoid weight (2 - delta_j0)/2
  that Eq. coeff folds in:
      D(E) = (tau / 2pi) [ w_0 C(0) + 2 Re sum_{j=1}^{N_t} w_j exp(i E t_j) C(t_j) ].
  The paper says a window is "typically employed" but names none; NONE (w_j = 1) and
  HANN (w_j = (1 + cos(pi j / (N_t + 1)))/2) are offered.
* Kernel-polynomial route (used for the moment-to-energy-grid reconstruction; the
  paper cites the KPM review of Weisse et al., Rev. Mod. Phys. 78, 275 (2006), Sec. II):
      D(E) = [ g_0 m_0 + 2 sum_{n=1}^{M-1} g_n Re(m_n) T_n(E~) ] / (pi |H| sqrt(1 - E~^2)),
  E~ = (E - H0)/|H|, with the Jackson damping factors (Weisse et al. Eq. 71)
      g_n = [ (M - n + 1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1)) ] / (M + 1).

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import numpy as np

WINDOW_NONE, WINDOW_HANN = 0, 1


def window(n_steps: int, kind: int) -> np.ndarray:
    j = np.arange(n_steps + 1, dtype=np.float64)
    if kind == WINDOW_NONE:
        return np.ones(n_steps + 1)
    if kind == WINDOW_HANN:
        return 0.5 * (1.0 + np.cos(np.pi * j / (n_steps + 1)))
    raise ValueError("unknown window")


def dos_fourier(C: np.ndarray, tau_phys: float, energies: np.ndarray, window_kind: int = WINDOW_NONE) -> np.ndarray:
    """DOS on `energies` from C(t_j), j = 0..N_t, t_j = j tau_phys."""
    n_steps = C.size - 1
    w = window(n_steps, window_kind)
    out = np.empty(energies.size)
    for k, E in enumerate(np.asarray(energies, dtype=np.float64)):
        s = w[0] * C[0].real
        for j in range(1, n_steps + 1):
            s += 2.0 * (w[j] * np.exp(1j * E * j * tau_phys) * C[j]).real
        out[k] = tau_phys / (2.0 * np.pi) * s
    return out


def jackson_factors(M: int) -> np.ndarray:
    n = np.arange(M, dtype=np.float64)
    q = np.pi / (M + 1)
    return ((M - n + 1) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (M + 1)


def cheb_T(n_max: int, x: float) -> np.ndarray:
    """T_0(x)..T_{n_max-1}(x) for |x| <= 1 from the trigonometric definition cos(n arccos x)."""
    return np.cos(np.arange(n_max, dtype=np.float64) * np.arccos(x))


def dos_jackson(mu: np.ndarray, energies: np.ndarray, H0: float, half_width: float) -> np.ndarray:
    """Jackson-damped Chebyshev DOS on `energies` from moments mu[0..M-1]."""
    M = mu.size
    g = jackson_factors(M)
    out = np.zeros(energies.size)
    for k, E in enumerate(np.asarray(energies, dtype=np.float64)):
        x = (E - H0) / half_width
        if abs(x) >= 1.0:
            continue
        T = cheb_T(M, x)
        s = g[0] * mu[0].real + 2.0 * np.sum(g[1:] * mu[1:].real * T[1:])
        out[k] = s / (np.pi * half_width * np.sqrt(1.0 - x * x))
    return out
