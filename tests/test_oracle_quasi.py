"""Pins of the oracle's quasi-eigenstates (Sec. IV): the sequential form (Eq. form1_sequential)
and the energy-based concurrent form (Eqs. form2_concurrent, QE_coeff) against the closed form
from exact diagonalisation, |Psi(E)> = sum_k <k|psi> K(E - E_k) |k> with the sampled kernel
K(e) = (tau/2pi)[1 + 2 sum_{j=1}^{N_t} cos(e t_j)], and against each other."""
import math

import numpy as np
import pytest

from oracle import lattice, propagate as pr, quasi, spectra


@pytest.fixture(scope="module")
def honey():
    lat = lattice.build_lattice(lattice.HONEYCOMB, (8, 6, 1), t=-2.7, W=1.5, seed=17)
    psi = pr.random_phase_states(lat, 5, 1)[0]
    E, U = np.linalg.eigh(lat.H.toarray())
    return lat, psi, E, U


def ed_qe(lat, psi, E, U, energies, Nt):
    tau = math.pi / lat.half_width
    j = np.arange(1, Nt + 1) * tau
    ov = U.conj().T @ psi
    out = []
    for e in energies:
        K = tau / (2 * np.pi) * (1 + 2 * np.cos(np.outer(e - E, j)).sum(axis=1))
        out.append(U @ (ov * K))
    return np.array(out)


def test_quasi_eigenstates_match_exact_diagonalisation(honey):
    lat, psi, E, U = honey
    energies = np.array([-6.0, -2.7, -0.4, 0.0, 3.3, 7.9])
    Nt = 40
    ref = ed_qe(lat, psi, E, U, energies, Nt)
    seq = quasi.qe_sequential(lat, psi, energies, Nt)
    con = quasi.qe_concurrent_e(lat, psi, energies, Nt)
    assert np.max(np.abs(seq - ref)) < 1e-12
    assert np.max(np.abs(con - ref)) < 1e-12


def test_quasi_eigenstate_overlap_is_fourier_dos(honey):
    """<psi|Psi(E)> equals the unwindowed Fourier DOS of Sec. III (same samples, same weights)."""
    lat, psi, _, _ = honey
    energies = np.linspace(-8, 8, 9)
    Nt = 25
    con = quasi.qe_concurrent_e(lat, psi, energies, Nt)
    C = pr.correlation_sequential(lat, psi, Nt)
    D = spectra.dos_fourier(C, math.pi / lat.half_width, energies, spectra.WINDOW_NONE)
    assert np.max(np.abs(np.array([np.vdot(psi, v) for v in con]) - D)) < 1e-12


def test_qe_coefficients_real_and_drop_h0_shift():
    """C_n(E) depends on E - H0 only; shifting both leaves it unchanged."""
    a = quasi.qe_coefficients([0.3, -1.0], 12, math.pi, 0.0, 3.0, 60)
    b = quasi.qe_coefficients([1.3, 0.0], 12, math.pi, 1.0, 3.0, 60)
    assert np.max(np.abs(a - b)) < 1e-14
    assert a.dtype == np.float64
