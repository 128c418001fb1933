"""Quasi-eigenstates (Sec. IV) in the sequential and the energy-based concurrent form (FP64).

Definition (Eq. QE): |Psi(E)> = (1/2pi) int exp(iEt) |psi(t)> dt, i.e. form 1 (Eq. form1) with
a(E, t) = exp(iEt)/(2pi).  Discretised at t_j = j tau as in Eq. form1_sequential:
    |Psi(E)> = tau a(E,0)|psi> + tau sum_{j=1}^{N_t} [a(E,t_j)|psi(t_j)> + a(E,-t_j)|psi(-t_j)>],
with |psi(+-t_j)> propagated step by step forwards and backwards (QE-Sequential).

Energy-based concurrent form (Eqs. form2_concurrent, QE_coeff):
    |Psi(E)> = sum_{n < N(t~_tot)} C_n(E) T_n(H~)|psi>,
    C_n(E) = tau sum_{j=0}^{N_t} ((2 - delta_j0)/2) [a(E,t_j) c_n(t~_j) e^{-i H0 t_j} + a(E,-t_j) c_n(-t~_j) e^{i H0 t_j}].
The printed Eq. QE_coeff omits the 1/(2pi) of Eq. QE; the reading used keeps it (a(E,t) as above).
The phase exp(-+ i H0 t) completes exp(-iHt) = exp(-iH0 t) exp(-iH~ t~) (H0 = 0 in the paper).
With c_n(-t~) = conj(c_n(t~)) the coefficient is real:
    C_0(E) = (tau/2pi) sum_j w_j 2 J_0(t~_j) cos(eps t_j),
    C_n(E) = (tau/2pi) sum_j w_j 4 J_n(t~_j) Re[(-i)^n exp(i eps t_j)],   eps = E - H0,  n >= 1.

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .bessel import bessel_j_sequence, truncation_order
from .lattice import Lattice
from .propagate import chebyshev_states, evolve_step


def qe_sequential(lat: Lattice, psi: np.ndarray, energies, n_steps: int, tau: float = np.pi) -> np.ndarray:
    """[n_E, N] quasi-eigenstates by forward and backward step-by-step propagation."""
    energies = np.asarray(energies, dtype=np.float64)
    tphys = tau / lat.half_width
    out = np.outer(np.full(energies.size, tphys / (2 * np.pi)), psi).astype(np.complex128)
    fwd = psi.astype(np.complex128)
    bwd = psi.astype(np.complex128)
    for j in range(1, n_steps + 1):
        fwd = evolve_step(lat, fwd, tau)
        bwd = evolve_step(lat, bwd, -tau)
        t = j * tphys
        out += (tphys / (2 * np.pi)) * (np.exp(1j * energies * t)[:, None] * fwd[None, :]
                                        + np.exp(-1j * energies * t)[:, None] * bwd[None, :])
    return out


def qe_coefficients(energies, n_steps: int, tau: float, H0: float, half_width: float, n_terms: int) -> np.ndarray:
    """[n_E, n_terms] real C_n(E) of the energy-based form (Eq. QE_coeff with a = e^{iEt}/2pi)."""
    energies = np.asarray(energies, dtype=np.float64)
    tphys = tau / half_width
    C = np.zeros((energies.size, n_terms))
    for j in range(0, n_steps + 1):
        w = 0.5 if j == 0 else 1.0
        J = bessel_j_sequence(j * tau, n_terms - 1) if j else np.eye(1, n_terms)[0]
        phase = np.exp(1j * (energies - H0) * j * tphys)           # e^{i eps t_j}
        n = np.arange(n_terms)
        rot = (-1j) ** (n % 4)                                     # (-i)^n
        term = 4.0 * (rot[None, :] * phase[:, None]).real * J[None, :]
        term[:, 0] = 2.0 * J[0] * phase.real
        C += w * term
    return C * tphys / (2 * np.pi)


def qe_concurrent_e(lat: Lattice, psi: np.ndarray, energies, n_steps: int, tau: float = np.pi) -> np.ndarray:
    """[n_E, N] quasi-eigenstates from one Chebyshev recurrence with C_n(E)."""
    n_terms = truncation_order(n_steps * tau)
    C = qe_coefficients(energies, n_steps, tau, lat.H0, lat.half_width, n_terms)
    out = np.zeros((C.shape[0], psi.size), dtype=np.complex128)
    for n, phi in enumerate(chebyshev_states(lat, psi, n_terms)):
        out += C[:, n][:, None] * phi[None, :]
    return out
