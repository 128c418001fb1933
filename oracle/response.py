"""Fermi-Dirac filtered response functions (FP64): optical conductivity (Sec. on OC) and dynamical
polarization (Sec. on DP), in the sequential form, plus the Fermi-Dirac operator itself.

Definitions followed (hbar = e = k_B = 1):
* Fermi-Dirac operator f(H) = [1 + exp((H - mu)/kT)]^{-1}, applied exactly through the
  eigen-decomposition of H (plain definition; small lattices only), or as its Chebyshev series
  sum_n a_n T_n(H~) with a_n from Chebyshev-Gauss quadrature on K nodes,
      a_n = ((2 - delta_n0)/K) sum_k f(H0 + |H| cos th_k) cos(n th_k),  th_k = pi (k + 1/2)/K
  (the expansion the library evaluates; pinned against the exact operator).
* OC correlation (Eq. oc_corr): C(t) = <psi_1(t)| J_a |psi_2(t)>,
      psi_1(t) = e^{-iHt} f(H) psi,  psi_2(t) = e^{-iHt} [1 - f(H)] J_b psi,
  sampled at t_j = j tau, tau~ = pi/2, both states propagated step by step (OC-Sequential).
* Re sigma_ab(w) = 2 (e^{-w/kT} - 1)/(w A) int_0^{t_tot} sin(w t) Im C(t) dt (the Kubo form of the
  OC section), read with:
    - the trace: the correlation of one normalised random state estimates Tr[...]/N, so the
      sample's sum is N C(t) and, with A = N x (area per site), sigma = 2 (e^{-w/kT} - 1)/(w a_site)
      int sin(w t) Im C dt;
    - the limit E -> 0+ of the damping e^{-Et} taken as no damping on the finite window, with the
      trapezoid weights (2 - delta_j0)/2 and an optional Hann window (as for the DOS);
    - kT = 0 as the limit e^{-w/kT} = 0 (w > 0); w = 0 gives 0 (the Drude term is excluded).
* Im sigma from the Kramers-Kronig relation of the OC section with Re sigma even in w, on the
  uniform grid w_k = k dw:  Im sigma(w) = -(2w/pi) P int_0^inf Re sigma(w')/(w'^2 - w^2) dw',
  the principal value by Maclaurin's rule (every other node, weight 2 dw; the node w = 0 weight
  dw), which is exact to O(dw^2) for smooth Re sigma.
* DP correlation: C(t, q) = <psi_1(t)| rho(q) |psi_2(q, t)>, psi_1 as above,
  psi_2(q, t) = e^{-iHt} [1 - f(H)] rho(-q) psi, rho(q) = sum_i e^{i q.r_i} |i><i|;
  Pi(q, w) = -(2/A) int_0^{t_tot} e^{iwt} Im C(t, q) dt with the same trace reading
  (Pi = -(2/a_site) int e^{iwt} Im C dt), weights and window.
Site positions r_i: square and cubic lattices with unit spacing at (x, y, z); graphene
A(x,y) = x a1 + y a2, B(x,y) = A(x,y) + (1, 0), a1 = (3/2, sqrt3/2), a2 = (3/2, -sqrt3/2).

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import expit

from .conductivity import area_per_site, current_operator
from .lattice import Lattice, HONEYCOMB, CUBIC
from .propagate import chebyshev_states, evolve_step
from .spectra import window

SQ3 = math.sqrt(3.0)


def fermi(E, mu: float, kT: float) -> np.ndarray:
    """Occupation 1/(1 + e^{(E-mu)/kT}); kT = 0 is the step (1/2 at E = mu)."""
    E = np.asarray(E, dtype=np.float64)
    if kT == 0.0:
        return np.where(E < mu, 1.0, np.where(E > mu, 0.0, 0.5))
    return expit(-(E - mu) / kT)


def fermi_operator_exact(lat: Lattice, X: np.ndarray, mu: float, kT: float, power: float = 1.0) -> np.ndarray:
    """f(H)^power X through the eigen-decomposition of the dense H."""
    E, U = np.linalg.eigh(lat.H.toarray())
    g = fermi(E, mu, kT) ** power
    return U @ (g * (U.conj().T @ X))


def fermi_cheb_coefficients(mu: float, kT: float, H0: float, half_width: float, n_terms: int,
                            n_nodes: int, power: float = 1.0) -> np.ndarray:
    """a_n, n < n_terms, of f(H0 + |H| x)^power = sum_n a_n T_n(x) by Chebyshev-Gauss quadrature."""
    k = np.arange(n_nodes, dtype=np.float64)
    th = np.pi * (k + 0.5) / n_nodes
    fk = fermi(H0 + half_width * np.cos(th), mu, kT) ** power
    a = np.empty(n_terms)
    for n in range(n_terms):
        a[n] = (2.0 if n else 1.0) / n_nodes * np.sum(fk * np.cos(n * th))
    return a


def fermi_operator_cheb(lat: Lattice, X: np.ndarray, a: np.ndarray) -> np.ndarray:
    out = np.zeros_like(X, dtype=np.complex128)
    for n, phi in enumerate(chebyshev_states(lat, X, a.size)):
        out += a[n] * phi
    return out


def positions(lat: Lattice) -> np.ndarray:
    """[n_active, 3] site positions in the library's geometry."""
    Lx, Ly, Lz = lat.L
    full = np.flatnonzero(lat.active)
    if lat.kind == HONEYCOMB:
        s = full % 2
        c = full // 2
        x, y = c % Lx, c // Lx
        a1 = np.array([1.5, SQ3 / 2, 0.0])
        a2 = np.array([1.5, -SQ3 / 2, 0.0])
        return x[:, None] * a1 + y[:, None] * a2 + s[:, None] * np.array([1.0, 0.0, 0.0])
    if lat.kind == CUBIC:
        x = full % Lx
        y = (full // Lx) % Ly
        z = full // (Lx * Ly)
        return np.stack([x, y, z], axis=1).astype(np.float64)
    return np.stack([full % Lx, full // Lx, np.zeros(full.size)], axis=1).astype(np.float64)


def density_phases(lat: Lattice, q) -> np.ndarray:
    """Diagonal of rho(q): e^{i q.r_i}."""
    return np.exp(1j * (positions(lat) @ np.asarray(q, dtype=np.float64)))


def _propagate_pair(lat, psi1, psi2, n_steps, tau, inner):
    C = np.empty(n_steps + 1, dtype=np.complex128)
    for j in range(n_steps + 1):
        C[j] = inner(psi1, psi2)
        if j < n_steps:
            psi1 = evolve_step(lat, psi1, tau)
            psi2 = evolve_step(lat, psi2, tau)
    return C


def oc_correlation_sequential(lat: Lattice, psi: np.ndarray, alpha: int, beta: int, mu: float, kT: float,
                              n_steps: int, tau: float = np.pi / 2) -> np.ndarray:
    Ja = current_operator(lat, alpha)
    Jb = current_operator(lat, beta)
    psi1 = fermi_operator_exact(lat, psi.astype(np.complex128), mu, kT)
    Jpsi = Jb @ psi
    psi2 = Jpsi - fermi_operator_exact(lat, Jpsi, mu, kT)
    return _propagate_pair(lat, psi1, psi2, n_steps, tau, lambda a, b: np.vdot(a, Ja @ b))


def dp_correlation_sequential(lat: Lattice, psi: np.ndarray, q, mu: float, kT: float, n_steps: int,
                              tau: float = np.pi / 2) -> np.ndarray:
    ph = density_phases(lat, q)
    psi1 = fermi_operator_exact(lat, psi.astype(np.complex128), mu, kT)
    x = ph.conj() * psi
    psi2 = x - fermi_operator_exact(lat, x, mu, kT)
    return _propagate_pair(lat, psi1, psi2, n_steps, tau, lambda a, b: np.vdot(a, ph * b))


def _weights(n_steps: int, window_kind: int) -> np.ndarray:
    w = window(n_steps, window_kind).copy()
    w[0] *= 0.5
    return w


def oc_sigma_real(C: np.ndarray, omegas, kT: float, tau_phys: float, area: float, window_kind: int = 0) -> np.ndarray:
    omegas = np.asarray(omegas, dtype=np.float64)
    n_steps = C.size - 1
    t = np.arange(n_steps + 1) * tau_phys
    w = _weights(n_steps, window_kind)
    out = np.zeros(omegas.size)
    for k, om in enumerate(omegas):
        if om == 0.0:
            continue
        boltz = 0.0 if kT == 0.0 else math.exp(-om / kT)
        integral = tau_phys * np.sum(w * np.sin(om * t) * C.imag)
        out[k] = 2.0 * (boltz - 1.0) / (om * area) * integral
    return out


def kramers_kronig_imag(omegas, re: np.ndarray) -> np.ndarray:
    """Im sigma on the uniform grid w_k = k dw (k = 0..K-1) from the even Re sigma, by
    Maclaurin's rule for the principal value (nodes of the parity opposite to k, weight 2 dw;
    the node w = 0 stands for itself and its mirror image, weight dw)."""
    om = np.asarray(omegas, dtype=np.float64)
    K = om.size
    if K < 2:
        return np.zeros(K)
    dw = om[1] - om[0]
    if om[0] != 0.0 or np.max(np.abs(om - dw * np.arange(K))) > 1e-9 * max(1.0, om[-1]):
        raise ValueError("Kramers-Kronig needs the uniform grid w_k = k dw")
    re = np.asarray(re, dtype=np.float64)
    out = np.zeros(K)
    j = np.arange(K)
    wgt = np.where(j == 0, dw, 2.0 * dw)
    for k in range(K):
        sel = ((j - k) % 2) == 1
        den = om[sel] ** 2 - om[k] ** 2
        out[k] = -2.0 * om[k] / np.pi * np.sum(re[sel] * wgt[sel] / den)
    return out


def dp_polarization(C: np.ndarray, omegas, tau_phys: float, area: float, window_kind: int = 0) -> np.ndarray:
    omegas = np.asarray(omegas, dtype=np.float64)
    n_steps = C.size - 1
    t = np.arange(n_steps + 1) * tau_phys
    w = _weights(n_steps, window_kind)
    return np.array([-2.0 / area * tau_phys * np.sum(w * np.exp(1j * om * t) * C.imag) for om in omegas])


def lehmann_correlation(lat: Lattice, psi: np.ndarray, A_op, B_op, mu: float, kT: float, times) -> np.ndarray:
    """<psi| f e^{iHt} A e^{-iHt} (1-f) B |psi> from the eigen-decomposition (test pin)."""
    E, U = np.linalg.eigh(lat.H.toarray())
    f = fermi(E, mu, kT)
    Ad = U.conj().T @ (A_op @ U)
    Bpsi = U.conj().T @ (B_op @ psi)
    c = U.conj().T @ psi
    out = np.empty(len(times), dtype=np.complex128)
    for j, t in enumerate(times):
        bra = f * c * np.exp(-1j * E * t)       # coefficients of e^{-iHt} f psi
        ket = (1.0 - f) * Bpsi * np.exp(-1j * E * t)
        out[j] = np.vdot(bra, Ad @ ket)
    return out
