"""Pins of the Fermi-Dirac operator, the optical-conductivity and the dynamical-polarization
oracle (oracle/response.py) against closed forms and an independent eigen-decomposition."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import conductivity as oec, lattice as olat, propagate as oprop, response as R


def test_fermi_operator_on_plane_waves_is_the_occupation():
    """Clean periodic square lattice: |k> = e^{ik.r}/sqrt N has E(k) = 2t(cos kx + cos ky),
    so f(H)|k> = f(E(k))|k> (closed form, independent of the eigen-solver's basis)."""
    Lx, Ly, t = 8, 6, 1.0
    lat = olat.build_lattice(olat.SQUARE, (Lx, Ly, 1), t=t)
    r = R.positions(lat)
    mu, kT = 0.4, 0.3
    for mx, my in [(0, 0), (1, 2), (3, 5), (4, 3)]:
        k = np.array([2 * np.pi * mx / Lx, 2 * np.pi * my / Ly, 0.0])
        v = np.exp(1j * r @ k) / math.sqrt(Lx * Ly)
        E = 2 * t * (math.cos(k[0]) + math.cos(k[1]))
        f = 1.0 / (1.0 + math.exp((E - mu) / kT))
        out = R.fermi_operator_exact(lat, v, mu, kT)
        assert np.max(np.abs(out - f * v)) < 1e-13
        half = R.fermi_operator_exact(lat, v, mu, kT, power=0.5)
        assert np.max(np.abs(half - math.sqrt(f) * v)) < 1e-13


def test_fermi_chebyshev_series_matches_exact_operator():
    lat = olat.build_lattice(olat.HONEYCOMB, (6, 5, 1), t=-2.7, W=1.0, seed=3)
    psi = oprop.random_phase_states(lat, 4, 1)[0]
    for mu, kT, n in [(0.3, 0.2, 400), (-2.0, 0.5, 200)]:
        a = R.fermi_cheb_coefficients(mu, kT, lat.H0, lat.half_width, n, 4 * n)
        x = R.fermi_operator_cheb(lat, psi, a)
        y = R.fermi_operator_exact(lat, psi, mu, kT)
        assert np.max(np.abs(x - y)) < 1e-12
    # high temperature: f -> 1/2 identity
    a = R.fermi_cheb_coefficients(0.0, 1e6, lat.H0, lat.half_width, 8, 64)
    assert abs(a[0] - 0.5) < 1e-6 and np.max(np.abs(a[1:])) < 1e-5


def test_positions_reproduce_bond_vectors():
    """Interior bonds: r_j - r_i equals the current operator's bond vectors."""
    for kind, L in [(olat.HONEYCOMB, (5, 4, 1)), (olat.SQUARE, (5, 4, 1)), (olat.CUBIC, (4, 3, 5))]:
        lat = olat.build_lattice(kind, L, t=1.0, pbc=(0, 0, 0))
        r = R.positions(lat)
        bv = oec.bond_vectors(kind)
        full = np.flatnonzero(lat.active)
        for i in range(full.size):
            sub = full[i] % 2 if kind == olat.HONEYCOMB else 0
            for d in range(lat.nbr_full.shape[1]):
                j = lat.nbr_full[full[i], d]
                if j >= 0:
                    assert np.allclose(r[lat.compact[j]] - r[i], bv[sub, d], atol=1e-14)


@pytest.mark.parametrize("kind,L,W", [(olat.HONEYCOMB, (6, 5, 1), 1.0), (olat.SQUARE, (7, 6, 1), 1.5),
                                      (olat.CUBIC, (4, 3, 4), 1.0)])
def test_oc_correlation_equals_lehmann_form(kind, L, W):
    lat = olat.build_lattice(kind, L, t=1.0, W=W, seed=11)
    psi = oprop.random_phase_states(lat, 2, 1)[0]
    mu, kT, Nt = 0.2, 0.25, 15
    ts = np.arange(Nt + 1) * (np.pi / 2) / lat.half_width
    dims = 3 if kind == olat.CUBIC else 2
    for a in range(dims):
        for b in range(dims):
            C = R.oc_correlation_sequential(lat, psi, a, b, mu, kT, Nt)
            L_ = R.lehmann_correlation(lat, psi, oec.current_operator(lat, a), oec.current_operator(lat, b),
                                       mu, kT, ts)
            assert np.max(np.abs(C - L_)) < 1e-12 * max(1.0, np.max(np.abs(L_)))


def test_dp_correlation_equals_lehmann_form():
    lat = olat.build_lattice(olat.HONEYCOMB, (6, 5, 1), t=-2.7, W=0.5, vacancy_frac=0.05, seed=12)
    psi = oprop.random_phase_states(lat, 3, 1)[0]
    mu, kT, Nt = -0.5, 0.3, 12
    ts = np.arange(Nt + 1) * (np.pi / 2) / lat.half_width
    for q in ([0.2, -0.4, 0.0], [1.1, 0.3, 0.0]):
        ph = R.density_phases(lat, q)
        C = R.dp_correlation_sequential(lat, psi, q, mu, kT, Nt)
        L_ = R.lehmann_correlation(lat, psi, sp.diags(ph), sp.diags(ph.conj()), mu, kT, ts)
        assert np.max(np.abs(C - L_)) < 1e-12


def test_oc_and_dp_integrals_match_closed_forms():
    """C(t) = A e^{-i D t}: int_0^T sin(wt) Im C dt and int_0^T e^{iwt} Im C dt in closed form.
    The weights (2 - delta_j0)/2 give the end point full weight: the trapezoid integral plus
    tau/2 times the integrand at T."""
    A, D, T, n = 0.7, 1.3, 40.0, 40000
    tau = T / n
    t = np.arange(n + 1) * tau
    C = A * np.exp(-1j * D * t)
    kT, area = 0.4, 1.7
    for w in (0.5, 1.2, 2.9):
        exact = -A * (math.sin((w - D) * T) / (2 * (w - D)) - math.sin((w + D) * T) / (2 * (w + D)))
        exact += tau / 2 * math.sin(w * T) * (-A * math.sin(D * T))
        pref = 2 * (math.exp(-w / kT) - 1) / (w * area)
        got = R.oc_sigma_real(C, [w], kT, tau, area)[0]
        assert abs(got - pref * exact) < 1e-5 * abs(pref) * max(1.0, abs(exact))
        # e^{iwt} (-A sin Dt): -A/(2i) [ (e^{i(w+D)T}-1)/(i(w+D)) - (e^{i(w-D)T}-1)/(i(w-D)) ]
        ip = (np.exp(1j * (w + D) * T) - 1) / (1j * (w + D))
        im_ = (np.exp(1j * (w - D) * T) - 1) / (1j * (w - D))
        exact_dp = -A / (2j) * (ip - im_) + tau / 2 * np.exp(1j * w * T) * (-A * math.sin(D * T))
        got_dp = R.dp_polarization(C, [w], tau, area)[0]
        assert abs(got_dp - (-2 / area) * exact_dp) < 1e-5 * (2 / area) * max(1.0, abs(exact_dp))
    assert R.oc_sigma_real(C, [0.0], kT, tau, area)[0] == 0.0


def test_kramers_kronig_on_a_lorentzian():
    """i/(w + i g) is analytic in the upper half plane: Re = g/(w^2+g^2) gives Im = w/(w^2+g^2)
    (error: O(dw^2) plus the tail beyond the grid)."""
    g = 0.5
    om = np.linspace(0.0, 200.0, 8001)
    re = g / (om ** 2 + g ** 2)
    im = R.kramers_kronig_imag(om, re)
    for w in (0.3, 0.5, 1.0, 2.0, 7.0):
        k = int(round(w / (om[1] - om[0])))
        assert abs(im[k] - om[k] / (om[k] ** 2 + g ** 2)) < 1e-7
    with pytest.raises(ValueError):
        R.kramers_kronig_imag(np.array([0.1, 0.2, 0.4]), np.ones(3))


def test_oc_correlation_equals_lehmann_form_on_a_long_range_lattice():
    """The Kubo correlation of the optical conductivity on a long-range lattice (each bond its own
    vector in the current operator) against the eigen-decomposition form."""
    lat = olat.build_lattice(olat.HONEYCOMB, (5, 4, 1), t=-2.7, W=0.8, seed=21, cutoff=3.1, decay=0.5)
    psi = oprop.random_phase_states(lat, 2, 1)[0]
    mu, kT, Nt = 0.3, 0.4, 12
    ts = np.arange(Nt + 1) * (np.pi / 2) / lat.half_width
    for a, b in ((0, 0), (0, 1), (1, 1)):
        C = R.oc_correlation_sequential(lat, psi, a, b, mu, kT, Nt)
        L_ = R.lehmann_correlation(lat, psi, oec.current_operator(lat, a), oec.current_operator(lat, b), mu, kT, ts)
        assert np.max(np.abs(C - L_)) < 1e-12 * max(1.0, np.max(np.abs(L_)))
