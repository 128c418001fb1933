"""Fermi-Dirac operator, optical conductivity and dynamical polarization on the GPU against the
FP64 oracle (oracle/response.py: exact Fermi-Dirac operator by eigen-decomposition, sequential
propagation of both filtered states).

Norms: states max|d|/max|ref| per state; C(t) max_j|dC|/max_j|C|; spectra max_w|d|/max_w|ref|.
Complex128 <= 1e-10 (spectra 1e-9), complex64 <= 3e-5 (spectra 1e-4)."""
import numpy as np
import pytest

from oracle import conductivity as oec, lattice as olat, propagate as oprop, response as R

pytestmark = pytest.mark.gpu
TOL = {0: 3e-5, 1: 1e-10}
TOL_SPEC = {0: 1e-4, 1: 1e-9}


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


def _oracle_lattice(spec):
    L = tuple(spec["L"]) + (1,) * (3 - len(spec["L"]))
    return olat.build_lattice(spec["kind"], L, t=spec["t"], W=spec["W"],
                              vacancy_frac=spec.get("vacancy_frac", 0.0), seed=spec["seed"],
                              pbc=spec.get("pbc", (1, 1, 1)))


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


LATS = [
    ("honey12x10_W1", dict(kind=1, L=(12, 10), t=-2.7, W=1.0, seed=41)),
    ("square9x11_open", dict(kind=0, L=(9, 11), t=1.0, W=1.5, seed=42, pbc=(0, 1, 1))),
    ("honey14x9_vac", dict(kind=1, L=(14, 9), t=-2.7, W=2.0, vacancy_frac=0.04, seed=43)),
    ("cubic5x4x6", dict(kind=2, L=(5, 4, 6), t=1.0, W=1.0, seed=44)),
]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("sqrt_f", [0, 1])
@pytest.mark.parametrize("name,spec", LATS, ids=[c[0] for c in LATS])
def test_fermi_operator_matches_exact(capi, ctx, name, spec, sqrt_f, prec):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle_lattice(spec)
    S = 3
    mu = ol.H0 + 0.2 * (ol.E_max - ol.E_min) / 2
    kT = 0.05 * (ol.E_max - ol.E_min) / 2
    out = np.zeros((S, ol.n), np.complex64 if prec == 0 else np.complex128)
    capi.tbpm_fermi_apply(ctx, lat, capi.request(n_states=S, precision=prec, state_seed=9), mu, kT, sqrt_f, out)
    psi = oprop.random_phase_states(ol, 9, S)
    for s in range(S):
        ref = R.fermi_operator_exact(ol, psi[s], mu, kT, power=0.5 if sqrt_f else 1.0)
        assert _rel(out[s], ref) <= TOL[prec], (s, _rel(out[s], ref))
    capi.tbpm_lattice_destroy(lat)


OC_CASES = [
    ("honey12x10_xx", LATS[0][1], 2, 0, 0),
    ("honey12x10_xy", LATS[0][1], 1, 0, 1),
    ("square9x11_open_yy", LATS[1][1], 3, 1, 1),
    ("honey14x9_vac_yx", LATS[2][1], 2, 1, 0),
    ("cubic5x4x6_zz", LATS[3][1], 1, 2, 2),
]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("form,b", [(0, 0), (2, 5), (2, 0)])
@pytest.mark.parametrize("name,spec,S,alpha,beta", OC_CASES, ids=[c[0] for c in OC_CASES])
def test_optical_conductivity_matches_oracle(capi, ctx, name, spec, S, alpha, beta, form, b, prec):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle_lattice(spec)
    mu = ol.H0 - 0.1 * (ol.E_max - ol.E_min) / 2
    kT = 0.08 * (ol.E_max - ol.E_min) / 2
    Nt, nw = 21, 33
    wmax = 1.2 * (ol.E_max - ol.E_min)
    window = 1 if form == 2 else 0
    req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=6,
                       window=window)
    C = np.zeros((S, Nt + 1), np.complex128)
    sig = np.zeros((S, nw), np.complex128)
    capi.tbpm_optical_conductivity(ctx, lat, req, alpha, beta, mu, kT, wmax, nw, C, sig)
    psi = oprop.random_phase_states(ol, 6, S)
    om = np.linspace(0.0, wmax, nw)
    tphys = (np.pi / 2) / ol.half_width
    area = oec.area_per_site(ol.kind)
    for s in range(S):
        Cref = R.oc_correlation_sequential(ol, psi[s], alpha, beta, mu, kT, Nt)
        assert _rel(C[s], Cref) <= TOL[prec], ("C", s, _rel(C[s], Cref))
        re = R.oc_sigma_real(Cref, om, kT, tphys, area, window)
        im = R.kramers_kronig_imag(om, re)
        scale = np.max(np.abs(re))
        assert np.max(np.abs(sig[s].real - re)) <= TOL_SPEC[prec] * scale, ("Re", s)
        assert np.max(np.abs(sig[s].imag - im)) <= TOL_SPEC[prec] * max(scale, np.max(np.abs(im))), ("Im", s)
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("form,b", [(0, 0), (2, 4)])
@pytest.mark.parametrize("name,spec,S,q", [
    ("honey12x10", LATS[0][1], 2, (0.35, -0.2, 0.0)),
    ("honey14x9_vac", LATS[2][1], 1, (1.1, 0.4, 0.0)),
    ("cubic5x4x6", LATS[3][1], 2, (0.3, 0.5, -0.7)),
], ids=["honey12x10", "honey14x9_vac", "cubic5x4x6"])
def test_polarization_matches_oracle(capi, ctx, name, spec, S, q, form, b, prec):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle_lattice(spec)
    mu = ol.H0 + 0.15 * (ol.E_max - ol.E_min) / 2
    kT = 0.1 * (ol.E_max - ol.E_min) / 2
    Nt = 17
    om = np.linspace(0.0, ol.E_max - ol.E_min, 13)
    req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=7)
    C = np.zeros((S, Nt + 1), np.complex128)
    Pi = np.zeros((S, om.size), np.complex128)
    capi.tbpm_polarization(ctx, lat, req, q, mu, kT, om, C, Pi)
    psi = oprop.random_phase_states(ol, 7, S)
    tphys = (np.pi / 2) / ol.half_width
    for s in range(S):
        Cref = R.dp_correlation_sequential(ol, psi[s], q, mu, kT, Nt)
        assert _rel(C[s], Cref) <= TOL[prec], ("C", s, _rel(C[s], Cref))
        ref = R.dp_polarization(Cref, om, tphys, oec.area_per_site(ol.kind))
        assert _rel(Pi[s], ref) <= TOL_SPEC[prec], ("Pi", s, _rel(Pi[s], ref))
    capi.tbpm_lattice_destroy(lat)


def test_response_forms_agree_on_a_larger_lattice(capi, ctx):
    """Sequential and state-based OC on honeycomb 64x48 (complex64), and bitwise repeatability."""
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (64, 48), t=-2.7, W=0.5, seed=45))
    Nt, nw = 48, 65
    out = []
    for form, b in [(0, 0), (2, 16), (2, 16)]:
        req = capi.request(n_states=4, precision=0, form=form, n_steps=Nt, time_block=b, state_seed=3)
        C = np.zeros((4, Nt + 1), np.complex128)
        sig = np.zeros((4, nw), np.complex128)
        capi.tbpm_optical_conductivity(ctx, lat, req, 0, 0, 0.5, 0.2, 18.0, nw, C, sig)
        out.append((C, sig))
    assert np.array_equal(out[1][0], out[2][0]) and np.array_equal(out[1][1], out[2][1])
    assert _rel(out[1][0], out[0][0]) < 1e-4
    capi.tbpm_lattice_destroy(lat)


def test_response_rejects_invalid_requests(capi, ctx):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (8, 8), t=-2.7, seed=1))
    C = np.zeros((1, 5), np.complex128)
    sig = np.zeros((1, 4), np.complex128)
    ok = capi.request(n_states=1, n_steps=4, form=0)
    with pytest.raises(capi.TbpmError):   # kT = 0
        capi.tbpm_optical_conductivity(ctx, lat, ok, 0, 0, 0.0, 0.0, 5.0, 4, C, sig)
    with pytest.raises(capi.TbpmError):   # moment-based form is not defined for the OC
        capi.tbpm_optical_conductivity(ctx, lat, capi.request(n_states=1, n_steps=4, form=1), 0, 0, 0.0, 0.1,
                                       5.0, 4, C, sig)
    with pytest.raises(capi.TbpmError):   # z direction on a 2-D lattice
        capi.tbpm_optical_conductivity(ctx, lat, ok, 2, 0, 0.0, 0.1, 5.0, 4, C, sig)
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("form,b,Nt", [(0, 0, 9), (2, 4, 9), (2, 0, 11), (0, 0, 0)])
@pytest.mark.parametrize("name,spec", LATS, ids=[c[0] for c in LATS])
def test_charge_density_matches_oracle(capi, ctx, name, spec, form, b, Nt, prec):
    from oracle import charge as ocd
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle_lattice(spec)
    S = 2
    mu = ol.H0 - 0.25 * (ol.E_max - ol.E_min) / 2
    kT = 0.06 * (ol.E_max - ol.E_min) / 2
    rho = np.zeros((S, ol.n))
    capi.tbpm_charge_density(ctx, lat, capi.request(n_states=S, precision=prec, form=form, n_steps=Nt,
                                                    time_block=b, state_seed=11), mu, kT, rho)
    psi = oprop.random_phase_states(ol, 11, S)
    tau = ocd.cd_default_tau(ol, mu, kT)
    for s in range(S):
        ref = ocd.charge_density_sequential(ol, psi[s], mu, kT, Nt, tau)
        assert _rel(rho[s], ref) <= TOL[prec], (s, _rel(rho[s], ref))
    capi.tbpm_lattice_destroy(lat)


def test_passes_of_fewer_states_give_the_same_results(capi, ctx):
    """OC, DP and CD with the states split into passes of one and of two states (the memory
    control used on large lattices) agree with one pass of all states (complex128)."""
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (10, 8), t=-2.7, W=1.0, seed=46))
    S, Nt, nw = 3, 15, 17
    om = np.linspace(0.0, 9.0, 5)
    res = []
    for k in (0, 1, 2):
        capi.tbpm_set_pass_states(ctx, k)
        C = np.zeros((S, Nt + 1), np.complex128)
        sig = np.zeros((S, nw), np.complex128)
        capi.tbpm_optical_conductivity(ctx, lat, capi.request(n_states=S, precision=1, form=2, n_steps=Nt,
                                                              time_block=4, state_seed=5), 0, 1, 0.2, 0.3, 12.0,
                                       nw, C, sig)
        Cd = np.zeros((S, Nt + 1), np.complex128)
        Pi = np.zeros((S, om.size), np.complex128)
        capi.tbpm_polarization(ctx, lat, capi.request(n_states=S, precision=1, form=0, n_steps=Nt, state_seed=5),
                               (0.4, 0.1, 0.0), 0.2, 0.3, om, Cd, Pi)
        rho = np.zeros((S, 160))
        capi.tbpm_charge_density(ctx, lat, capi.request(n_states=S, precision=1, form=2, n_steps=Nt, time_block=4,
                                                        state_seed=5), 0.2, 0.3, rho)
        res.append((C, sig, Cd, Pi, rho))
    capi.tbpm_set_pass_states(ctx, 0)
    for k in (1, 2):
        for a, b in zip(res[k], res[0]):
            assert _rel(a, b) < 1e-12, k
    capi.tbpm_lattice_destroy(lat)
