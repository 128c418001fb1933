"""DC (electronic) conductivity, Sec. V, in the sequential and moment-based forms (FP64).

Definitions followed (hbar = e = 1):
* Current operator J_a = i [H, P_a], P_a = -sum_i r_{a,i} |i><i|, so for every bond i-j
      (J_a)_{ij} = -i H_ij (r_j - r_i)_a,
  with r_j - r_i the bond vector (the nearest image across periodic boundaries).
  Geometries (the paper's TBG has its own; these are the library's lattices): square and simple
  cubic with unit lattice constant; honeycomb as graphene with C-C distance 1, A(x,y) at
  x a1 + y a2, B(x,y) at x a1 + y a2 + delta, a1 = (3/2, sqrt3/2), a2 = (3/2, -sqrt3/2),
  delta = (1, 0).  Bond vectors from A(x,y): to B(x,y) delta, to B(x-1,y) delta - a1,
  to B(x,y-1) delta - a2.
* Correlation (Eq. dc_corr): C(t,E) = <psi| J e^{iHt} J |Psi(E)> / |<psi|Psi(E)>|, with
  |Psi(E)> the quasi-eigenstate of Sec. IV.  Sequential form: psi_1(t) = e^{-iHt} J|psi>,
  C(t_j,E) = <psi_1(t_j)|J Psi(E)> / |<psi|Psi(E)>|.  Moment form (Eq. dc_mom):
  m_n(E) = <J psi| T_n(H~) |J Psi(E)>,  C(t_j,E) = e^{i H0 t_j} sum_{n<N(j tau~)} c_n^*(j tau~) m_n(E) / |<psi|Psi(E)>|.
* Conductivity (Eq. DC): sigma(E) = D(E)/A int_0^{t_tot} Re[e^{-iEt} C(t,E)] dt with
  D(E) = N <psi|Psi(E)> (states per unit energy of the whole sample; <psi|Psi(E)> is the
  normalised DOS of Sec. III) and A the area (2-D) or volume (3-D) of the sample: 1 per site
  (square, cubic) or 3 sqrt3/4 per site (graphene).  The time integral uses the weights
  (2 - delta_j0)/2 of Eq. coeff on t_j = j tau.  The paper prints no normalisation beyond this;
  the reading above is the library's.

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .bessel import cheb_coefficients, truncation_order
from .lattice import Lattice, SQUARE, HONEYCOMB, CUBIC, long_range_bonds
from .propagate import chebyshev_states, evolve_step
from .quasi import qe_concurrent_e

SQ3 = math.sqrt(3.0)


def bond_vectors(kind: int) -> np.ndarray:
    """[2 sublattices, z, 3] bond vectors r_j - r_i in the fixed neighbour order."""
    if kind == SQUARE:
        v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]], float)
        return np.stack([v, v])
    if kind == CUBIC:
        v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
        return np.stack([v, v])
    a1 = np.array([1.5, SQ3 / 2, 0.0])
    a2 = np.array([1.5, -SQ3 / 2, 0.0])
    d = np.array([1.0, 0.0, 0.0])
    A = np.stack([d, d - a1, d - a2])
    return np.stack([A, -A])


def area_per_site(kind: int) -> float:
    return 3.0 * SQ3 / 4.0 if kind == HONEYCOMB else 1.0


def current_operator(lat: Lattice, direction: int) -> sp.csr_matrix:
    """J_a as a sparse [n, n] complex matrix on the active sites.  Long-range lattices: every
    bond (i, j, image R) contributes -i t(r) (r_j + R - r_i)_a, its own bond vector."""
    if getattr(lat, "cutoff", 0.0) > 0.0:
        full_idx = np.flatnonzero(lat.active)
        rows, cols, tv, dv = long_range_bonds(lat.kind, lat.L, lat.pbc, full_idx, lat.t, lat.cutoff, lat.decay,
                                              with_disp=True)
        J = sp.coo_matrix((-1j * tv * dv[:, direction], (rows, cols)), shape=(lat.n, lat.n)).tocsr()
        J.sum_duplicates()
        return J
    bv = bond_vectors(lat.kind)
    rows, cols, vals = [], [], []
    full_idx = np.flatnonzero(lat.active)
    sub = (full_idx % 2) if lat.kind == HONEYCOMB else np.zeros(full_idx.size, int)
    for d in range(lat.nbr_full.shape[1]):
        j = lat.nbr_full[full_idx, d]
        keep = j >= 0
        keep[keep] &= lat.active[j[keep]]
        comp = bv[sub[keep], d, direction]
        rows.append(lat.compact[full_idx[keep]])
        cols.append(lat.compact[j[keep]])
        vals.append(-1j * lat.t * comp)
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(lat.n, lat.n)).tocsr()
    J.sum_duplicates()
    return J


def ec_correlation_sequential(lat, psi, energies, n_steps, direction=0, tau=np.pi):
    """[n_E, n_steps+1] C(t_j, E) by step-by-step propagation of J|psi>."""
    J = current_operator(lat, direction)
    qe = qe_concurrent_e(lat, psi, energies, n_steps, tau)
    ket = np.array([J @ v for v in qe])
    norm = np.abs(qe.conj() @ psi)
    psi1 = J @ psi
    C = np.empty((len(energies), n_steps + 1), dtype=np.complex128)
    for j in range(n_steps + 1):
        C[:, j] = (ket @ psi1.conj()) / norm
        if j < n_steps:
            psi1 = evolve_step(lat, psi1, tau)
    return C, qe


def ec_moments(lat, psi, energies, n_steps, direction=0, tau=np.pi):
    """m_n(E) = <J psi|T_n(H~)|J Psi(E)>, n < N(n_steps tau~)."""
    J = current_operator(lat, direction)
    qe = qe_concurrent_e(lat, psi, energies, n_steps, tau)
    ket = np.array([J @ v for v in qe])
    n_terms = truncation_order(n_steps * tau)
    m = np.empty((len(energies), n_terms), dtype=np.complex128)
    for n, phi in enumerate(chebyshev_states(lat, J @ psi, n_terms)):
        m[:, n] = ket @ phi.conj()
    return m, qe


def ec_correlation_from_moments(lat, m, qe, psi, n_steps, tau=np.pi):
    norm = np.abs(qe.conj() @ psi)
    C = np.empty((m.shape[0], n_steps + 1), dtype=np.complex128)
    for j in range(n_steps + 1):
        tj = j * tau
        nj = truncation_order(tj) if j else 1
        c = cheb_coefficients(tj, nj) if j else np.array([1.0 + 0j])
        C[:, j] = np.exp(1j * lat.H0 * tj / lat.half_width) * (m[:, :nj] @ c.conj()) / norm
    return C


def conductivity(lat, psi, energies, C, qe, tau=np.pi):
    """sigma(E_k) from C(t_j, E_k) (Eq. DC)."""
    energies = np.asarray(energies, float)
    tphys = tau / lat.half_width
    n_steps = C.shape[1] - 1
    w = np.ones(n_steps + 1)
    w[0] = 0.5
    t = np.arange(n_steps + 1) * tphys
    integral = tphys * np.sum(w[None, :] * (np.exp(-1j * np.outer(energies, t)) * C).real, axis=1)
    D = lat.n * (qe.conj() @ psi).real
    A = lat.n * area_per_site(lat.kind)
    return D / A * integral
