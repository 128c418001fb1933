"""Pins of the charge-density oracle (oracle/charge.py): the eigen-decomposition form of the
time average, norm conservation, the N_t = 0 estimate and the ensemble mean <r|f(H)|r>."""
import numpy as np

from oracle import charge as ocd, lattice as olat, propagate as oprop, response as R


def test_time_average_equals_lehmann_form():
    for kind, L in [(olat.HONEYCOMB, (6, 5, 1)), (olat.SQUARE, (7, 6, 1)), (olat.CUBIC, (4, 3, 4))]:
        lat = olat.build_lattice(kind, L, t=1.0, W=1.0, seed=21)
        psi = oprop.random_phase_states(lat, 5, 1)[0]
        mu, kT = lat.H0 - 0.3, 0.2
        tau = ocd.cd_default_tau(lat, mu, kT)
        rho = ocd.charge_density_sequential(lat, psi, mu, kT, 13, tau)
        ref = ocd.charge_density_lehmann(lat, psi, mu, kT, 13, tau)
        assert np.max(np.abs(rho - ref)) < 1e-12 * np.max(np.abs(ref))


def test_total_charge_is_conserved_and_zero_steps_is_plain_estimate():
    lat = olat.build_lattice(olat.HONEYCOMB, (8, 6, 1), t=-2.7, W=1.5, vacancy_frac=0.05, seed=22)
    psi = oprop.random_phase_states(lat, 6, 1)[0]
    mu, kT = 0.4, 0.3
    phi = R.fermi_operator_exact(lat, psi, mu, kT, power=0.5)
    total = lat.n * np.vdot(phi, phi).real
    for Nt in (0, 1, 9):
        rho = ocd.charge_density_sequential(lat, psi, mu, kT, Nt)
        assert abs(rho.sum() - total) < 1e-11 * total
    rho0 = ocd.charge_density_sequential(lat, psi, mu, kT, 0)
    assert np.max(np.abs(rho0 - lat.n * np.abs(phi) ** 2)) < 1e-13


def test_ensemble_mean_approaches_diagonal_of_fermi_operator():
    """Averaged over random states (and time), rho_i estimates <i|f(H)|i> (statistical pin:
    64 states, error well inside 5 standard errors)."""
    lat = olat.build_lattice(olat.SQUARE, (6, 6, 1), t=1.0, W=2.0, seed=23)
    mu, kT = 0.2, 0.25
    E, U = np.linalg.eigh(lat.H.toarray())
    exact = (np.abs(U) ** 2) @ R.fermi(E, mu, kT)
    samples = np.array([ocd.charge_density_sequential(lat, oprop.random_phase_states(lat, 100 + k, 1)[0],
                                                      mu, kT, 40) for k in range(64)])
    mean = samples.mean(axis=0)
    se = samples.std(axis=0, ddof=1) / np.sqrt(samples.shape[0])
    assert np.all(np.abs(mean - exact) < 5 * se + 1e-12)
    assert abs(mean.sum() - exact.sum()) < 0.05 * exact.sum()
