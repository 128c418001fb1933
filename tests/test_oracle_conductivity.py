"""Pins of the oracle's DC conductivity (Sec. V): the current operator against the commutator
J = i[H, P] on open lattices (where positions are single-valued), the sequential and moment
forms against each other and against a dense exact-diagonalisation evaluation of Eq. dc_corr."""
import math

import numpy as np
import pytest

from oracle import lattice, propagate as pr, conductivity as ec


def positions(lat):
    """Real-space positions of the active sites (open lattices: no wrapping)."""
    full = np.flatnonzero(lat.active)
    Lx, Ly, Lz = lat.L
    if lat.kind == lattice.HONEYCOMB:
        s, c = full % 2, full // 2
        x, y = c % Lx, c // Lx
        a1 = np.array([1.5, math.sqrt(3) / 2, 0])
        a2 = np.array([1.5, -math.sqrt(3) / 2, 0])
        return x[:, None] * a1 + y[:, None] * a2 + s[:, None] * np.array([1.0, 0, 0])
    if lat.kind == lattice.SQUARE:
        return np.stack([full % Lx, full // Lx, np.zeros(full.size)], axis=1).astype(float)
    return np.stack([full % Lx, (full // Lx) % Ly, full // (Lx * Ly)], axis=1).astype(float)


@pytest.mark.parametrize("kind,L", [(lattice.SQUARE, (5, 4, 1)), (lattice.HONEYCOMB, (4, 3, 1)),
                                    (lattice.CUBIC, (3, 3, 4))])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_current_operator_is_commutator_on_open_lattices(kind, L, direction):
    lat = lattice.build_lattice(kind, L, t=-1.3, W=0.8, seed=2, pbc=(0, 0, 0))
    J = ec.current_operator(lat, direction).toarray()
    P = -np.diag(positions(lat)[:, direction])
    H = lat.H.toarray()
    assert np.max(np.abs(J - 1j * (H @ P - P @ H))) < 1e-13


def test_correlation_forms_and_exact_diagonalisation():
    lat = lattice.build_lattice(lattice.HONEYCOMB, (6, 5, 1), t=-2.7, W=1.0, seed=3)
    psi = pr.random_phase_states(lat, 1, 1)[0]
    E = np.array([-3.0, 0.5, 2.2])
    Nt = 20
    Cs, qe = ec.ec_correlation_sequential(lat, psi, E, Nt)
    m, qe2 = ec.ec_moments(lat, psi, E, Nt)
    Cm = ec.ec_correlation_from_moments(lat, m, qe2, psi, Nt)
    assert np.max(np.abs(Cs - Cm)) < 1e-11
    H = lat.H.toarray()
    J = ec.current_operator(lat, 0).toarray()
    Ek, U = np.linalg.eigh(H)
    tau = math.pi / lat.half_width
    Jpsi = J @ psi
    for j in (0, 7, 20):
        eiHt = U @ np.diag(np.exp(1j * Ek * j * tau)) @ U.conj().T
        for k in range(E.size):
            ref = np.vdot(Jpsi, eiHt @ (J @ qe[k])) / abs(np.vdot(psi, qe[k]))
            assert abs(Cs[k, j] - ref) < 1e-11


@pytest.mark.parametrize("kind,L,cutoff", [(lattice.HONEYCOMB, (5, 4, 1), 3.1), (lattice.SQUARE, (6, 5, 1), 2.9),
                                           (lattice.CUBIC, (4, 3, 3), 1.8)])
def test_long_range_current_operator_is_commutator_on_open_lattices(kind, L, cutoff):
    """Without periodic images every bond vector is r_j - r_i, so J_a = i[H, P_a] exactly."""
    lat = lattice.build_lattice(kind, L, t=-1.3, W=0.8, seed=2, pbc=(0, 0, 0), cutoff=cutoff, decay=0.6)
    H = lat.H.toarray()
    for direction in range(3 if kind == lattice.CUBIC else 2):
        J = ec.current_operator(lat, direction).toarray()
        P = -np.diag(positions(lat)[:, direction])
        assert np.max(np.abs(J - 1j * (H @ P - P @ H))) < 1e-13
