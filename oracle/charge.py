"""Charge density (CD section, Eq. rho) in the sequential form (FP64).

Definition followed: rho(r) = (N/2pi) int |<r| e^{-iHt} f^{1/2}(H) |psi>|^2 dt.  For a finite sample
the integrand does not decay (its zero-frequency part is the diagonal ensemble
sum_n |<r|n>|^2 |<n|f^{1/2} psi>|^2, whose mean over random states is <r|f(H)|r>/N), so the
integral is read as N times the time average of the integrand over the sampled window:
    rho_i = N sum_{j=0}^{N_t} w_j |psi(t_j)_i|^2 / sum_j w_j,  psi(t) = e^{-iHt} f^{1/2}(H) psi,
with w_j = (2 - delta_j0)/2 on t_j = j tau.  With N_t = 0 it is the plain stochastic estimate
N |<r|f^{1/2}|psi>|^2.  Time step: the integrand's frequencies are differences of occupied
energies, a band of width 2 Delta_occ, so tau = pi/Delta_occ (tau~ = pi|H|/Delta_occ), with the
occupied width read as Delta_occ = min(E_max, mu + 20 kT) - E_min (f^{1/2} < 5e-5 above).

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice
from .propagate import evolve_step
from .response import fermi_operator_exact


def cd_default_tau(lat: Lattice, mu: float, kT: float) -> float:
    """Rescaled time step pi |H| / Delta_occ."""
    occ = min(lat.E_max, mu + 20.0 * kT) - lat.E_min
    if occ <= 0:
        raise ValueError("no occupied states")
    return np.pi * lat.half_width / occ


def charge_density_sequential(lat: Lattice, psi: np.ndarray, mu: float, kT: float, n_steps: int,
                              tau: float | None = None) -> np.ndarray:
    """rho_i (length N) from one random state."""
    if tau is None:
        tau = cd_default_tau(lat, mu, kT)
    cur = fermi_operator_exact(lat, psi.astype(np.complex128), mu, kT, power=0.5)
    z = np.zeros(lat.n)
    wsum = 0.0
    for j in range(n_steps + 1):
        w = 0.5 if j == 0 else 1.0
        z += w * np.abs(cur) ** 2
        wsum += w
        if j < n_steps:
            cur = evolve_step(lat, cur, tau)
    return lat.n * z / wsum


def charge_density_lehmann(lat: Lattice, psi: np.ndarray, mu: float, kT: float, n_steps: int, tau: float) -> np.ndarray:
    """The same average from the eigen-decomposition: sum_{n,m} c_n c_m^* <r|n><m|r> avg_j e^{-i(E_n-E_m)t_j}
    (test pin)."""
    E, U = np.linalg.eigh(lat.H.toarray())
    from .response import fermi
    c = np.sqrt(fermi(E, mu, kT)) * (U.conj().T @ psi)
    tphys = tau / lat.half_width
    j = np.arange(n_steps + 1)
    w = np.where(j == 0, 0.5, 1.0)
    dE = E[:, None] - E[None, :]
    avg = np.tensordot(w, np.exp(-1j * np.multiply.outer(j * tphys, dE)), axes=1) / w.sum()
    A = U * c[None, :]                         # A[r, n] = <r|n> c_n
    return lat.n * np.real(np.einsum("rn,nm,rm->r", A, avg, A.conj()))
