"""The state-based forms on honeycomb lattices wide enough for the register sweep's window pass
(four Chebyshev terms of a time block per pass into the block's buffer slots): quasi-eigenstates,
DC conductivity and optical conductivity in their sequential and time-block forms, complex64,
against the FP64 oracle with the tolerances of the smaller-lattice tests.  The lattices are the
smallest the window pass takes for the padded state count (band of 128 / (S/2) cells, 32 rows)."""
import numpy as np
import pytest

from oracle import conductivity as oec, lattice as olat, propagate as oprop, quasi as oqe, response as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_17432_gb300 import capi as c
    return c


@pytest.fixture(scope="module")
def ctx(capi):
    h = capi.tbpm_create(0)
    yield h
    capi.tbpm_destroy(h)


def _lattice(capi, ctx, spec):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = olat.build_lattice(spec["kind"], tuple(spec["L"]) + (1,), t=spec["t"], W=spec["W"], seed=spec["seed"],
                            pbc=spec.get("pbc", (1, 1, 1)))
    return lat, ol


QE_SPEC = dict(kind=1, L=(64, 40), t=-2.7, W=1.5, seed=51)  # 4 states: band of 64 cells


@pytest.mark.parametrize("form,b", [(0, 0), (2, 5), (2, 0)])
def test_quasi_eigenstates_through_window_passes(capi, ctx, form, b):
    lat, ol = _lattice(capi, ctx, QE_SPEC)
    S, Nt = 4, 23
    E = np.array([-5.0, -1.1, 0.0, 0.7, 4.2])
    out = np.zeros((E.size, S, ol.n), np.complex64)
    capi.tbpm_quasi_eigenstates(ctx, lat, capi.request(n_states=S, precision=0, form=form, n_steps=Nt,
                                                       time_block=b, state_seed=8), E, out)
    psi = oprop.random_phase_states(ol, 8, S)
    for s in (0, S - 1):
        ref = oqe.qe_concurrent_e(ol, psi[s], E, Nt)
        for k in range(E.size):
            err = np.max(np.abs(out[k, s] - ref[k])) / np.max(np.abs(ref[k]))
            assert err <= 1e-5, (form, b, s, k, err)
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("form,b", [(0, 0), (2, 4), (2, 0)])
def test_conductivity_through_window_passes(capi, ctx, form, b):
    lat, ol = _lattice(capi, ctx, QE_SPEC)
    S, Nt, direction = 4, 15, 0
    E = ol.H0 + np.array([-0.6, 0.05, 0.4]) * (ol.E_max - ol.E_min) / 2
    C = np.zeros((S, E.size, Nt + 1), np.complex128)
    sigma = np.zeros((S, E.size))
    capi.tbpm_conductivity(ctx, lat, capi.request(n_states=S, precision=0, form=form, n_steps=Nt, time_block=b,
                                                  state_seed=12), direction, E, C, sigma)
    psi = oprop.random_phase_states(ol, 12, S)
    for s in (0, S - 1):
        Cref, qe = oec.ec_correlation_sequential(ol, psi[s], E, Nt, direction)
        sref = oec.conductivity(ol, psi[s], E, Cref, qe)
        Dn = np.abs((qe.conj() @ psi[s]).real) / oec.area_per_site(ol.kind)
        for k in range(E.size):
            err = np.max(np.abs(C[s, k] - Cref[k])) / np.max(np.abs(Cref[k]))
            assert err <= 3e-5, ("C", s, k, err)
            bound = Dn[k] * (np.pi / ol.half_width) * np.sum(np.abs(Cref[k]))
            assert abs(sigma[s, k] - sref[k]) <= 3e-5 * bound, ("sigma", s, k)
    capi.tbpm_lattice_destroy(lat)


def test_conductivity_moment_form_through_window_passes(capi, ctx):
    """Concurrent-M form: the moments m_n(E) of J psi take four Chebyshev terms per window pass
    into the buffered slots; compared with the oracle's moment form term by term of C(t, E)."""
    lat, ol = _lattice(capi, ctx, QE_SPEC)
    S, Nt, direction = 4, 15, 1
    E = ol.H0 + np.array([-0.6, 0.05, 0.4]) * (ol.E_max - ol.E_min) / 2
    C = np.zeros((S, E.size, Nt + 1), np.complex128)
    sigma = np.zeros((S, E.size))
    capi.tbpm_conductivity(ctx, lat, capi.request(n_states=S, precision=0, form=1, n_steps=Nt, state_seed=13),
                           direction, E, C, sigma)
    psi = oprop.random_phase_states(ol, 13, S)
    for s in (0, S - 1):
        m, qe = oec.ec_moments(ol, psi[s], E, Nt, direction)
        Cref = oec.ec_correlation_from_moments(ol, m, qe, psi[s], Nt)
        for k in range(E.size):
            err = np.max(np.abs(C[s, k] - Cref[k])) / np.max(np.abs(Cref[k]))
            assert err <= 3e-5, ("C", s, k, err)
    capi.tbpm_lattice_destroy(lat)


OC_SPEC = dict(kind=1, L=(48, 32), t=-2.7, W=1.0, seed=52)  # 4 states: a pair block of 8, band of 32 cells


@pytest.mark.parametrize("form,b", [(0, 0), (2, 5)])
def test_optical_conductivity_through_window_passes(capi, ctx, form, b):
    lat, ol = _lattice(capi, ctx, OC_SPEC)
    S, Nt, nw, alpha, beta = 4, 21, 33, 0, 1
    mu = ol.H0 - 0.1 * (ol.E_max - ol.E_min) / 2
    kT = 0.08 * (ol.E_max - ol.E_min) / 2
    wmax = 1.2 * (ol.E_max - ol.E_min)
    C = np.zeros((S, Nt + 1), np.complex128)
    sig = np.zeros((S, nw), np.complex128)
    capi.tbpm_optical_conductivity(ctx, lat, capi.request(n_states=S, precision=0, form=form, n_steps=Nt,
                                                          time_block=b, state_seed=6), alpha, beta, mu, kT, wmax,
                                   nw, C, sig)
    psi = oprop.random_phase_states(ol, 6, S)
    for s in (0, S - 1):
        Cref = R.oc_correlation_sequential(ol, psi[s], alpha, beta, mu, kT, Nt)
        assert np.max(np.abs(C[s] - Cref)) / np.max(np.abs(Cref)) <= 3e-5, s
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("sqrt_f", [0, 1])
def test_fermi_operator_through_window_passes(capi, ctx, sqrt_f):
    """The Fermi-Dirac series (its buffered terms through the window passes) against the exact
    operator from the eigen-decomposition."""
    lat, ol = _lattice(capi, ctx, QE_SPEC)
    S = 4
    mu = ol.H0 + 0.2 * (ol.E_max - ol.E_min) / 2
    kT = 0.05 * (ol.E_max - ol.E_min) / 2
    out = np.zeros((S, ol.n), np.complex64)
    capi.tbpm_fermi_apply(ctx, lat, capi.request(n_states=S, precision=0, state_seed=9), mu, kT, sqrt_f, out)
    psi = oprop.random_phase_states(ol, 9, S)
    for s in (0, S - 1):
        ref = R.fermi_operator_exact(ol, psi[s], mu, kT, power=0.5 if sqrt_f else 1.0)
        assert np.max(np.abs(out[s] - ref)) / np.max(np.abs(ref)) <= 3e-5, s
    capi.tbpm_lattice_destroy(lat)
