"""Electronic conductivity on the GPU (Sec. V) in the sequential, state-based (EC-Concurrent-S) and
moment-based (EC-Concurrent-M) forms against the FP64 oracle (oracle/conductivity.py).

Norms: C(t_j, E) per energy, max_j |C_gpu - C_oracle| / max_j |C_oracle|; sigma(E) against the
bound |D/A| tau sum_j |C_j| of its own sum.  Complex128 <= 1e-10, complex64 <= 3e-5 (FP32
states through the quasi-eigenstate, the current operator and the propagation)."""
import numpy as np
import pytest

from oracle import conductivity as oec, lattice as olat, propagate as oprop

pytestmark = pytest.mark.gpu
TOL = {0: 3e-5, 1: 1e-10}


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


def _check(ol, psi_all, E, Nt, direction, C, sigma, prec, S):
    for s in range(S):
        Cref, qe = oec.ec_correlation_sequential(ol, psi_all[s], E, Nt, direction)
        sref = oec.conductivity(ol, psi_all[s], E, Cref, qe)
        tphys = np.pi / ol.half_width
        Dn = np.abs((qe.conj() @ psi_all[s]).real) / oec.area_per_site(ol.kind)
        for k in range(E.size):
            err = np.max(np.abs(C[s, k] - Cref[k])) / np.max(np.abs(Cref[k]))
            assert err <= TOL[prec], ("C", s, k, err)
            bound = Dn[k] * tphys * np.sum(np.abs(Cref[k]))
            assert abs(sigma[s, k] - sref[k]) <= TOL[prec] * bound, ("sigma", s, k, sigma[s, k], sref[k])


CASES = [
    ("honey12x10_W1", dict(kind=1, L=(12, 10), t=-2.7, W=1.0, seed=31), 2, 0),
    ("honey12x10_W1_y", dict(kind=1, L=(12, 10), t=-2.7, W=1.0, seed=31), 1, 1),
    ("square9x11_open", dict(kind=0, L=(9, 11), t=1.0, W=1.5, seed=32, pbc=(0, 1, 1)), 3, 0),
    ("honey14x9_vac", dict(kind=1, L=(14, 9), t=-2.7, W=2.0, vacancy_frac=0.04, seed=33), 2, 1),
    ("cubic5x4x6_z", dict(kind=2, L=(5, 4, 6), t=1.0, W=1.0, seed=34), 1, 2),
]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("form,b", [(0, 0), (2, 4), (2, 0), (1, 0)])
@pytest.mark.parametrize("name,spec,S,direction", CASES, ids=[c[0] for c in CASES])
def test_conductivity_matches_oracle(capi, ctx, name, spec, S, direction, form, b, prec):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle_lattice(spec)
    E = ol.H0 + np.array([-0.7, -0.2, 0.05, 0.45]) * (ol.E_max - ol.E_min) / 2
    Nt = 19
    req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=12)
    C = np.zeros((S, E.size, Nt + 1), np.complex128)
    sigma = np.zeros((S, E.size))
    capi.tbpm_conductivity(ctx, lat, req, direction, E, C, sigma)
    psi = oprop.random_phase_states(ol, 12, S)
    _check(ol, psi, E, Nt, direction, C, sigma, prec, S)
    capi.tbpm_lattice_destroy(lat)


def test_conductivity_many_energies_state_based_quasi_eigenstates(capi, ctx):
    """More than 200 energies switch the quasi-eigenstates to the state-based form."""
    spec = dict(kind=1, L=(6, 5), t=-2.7, W=1.0, seed=35)
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle_lattice(spec)
    E = np.linspace(-7.5, 7.5, 203)
    Nt = 9
    req = capi.request(n_states=1, precision=1, form=1, n_steps=Nt, state_seed=5)
    C = np.zeros((1, E.size, Nt + 1), np.complex128)
    sigma = np.zeros((1, E.size))
    capi.tbpm_conductivity(ctx, lat, req, 0, E, C, sigma)
    psi = oprop.random_phase_states(ol, 5, 1)
    _check(ol, psi, E, Nt, 0, C, sigma, 1, 1)
    capi.tbpm_lattice_destroy(lat)


def test_conductivity_forms_agree_and_repeat_bitwise(capi, ctx):
    """EC-Sequential, EC-Concurrent-S and EC-Concurrent-M on a larger lattice (complex64),
    and two identical calls give identical bits."""
    spec = dict(kind=1, L=(96, 64), t=-2.7, W=0.5, seed=36)
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    E = np.linspace(-6, 6, 9)
    Nt = 64
    out = {}
    for form, b in [(0, 0), (2, 16), (1, 0)]:
        req = capi.request(n_states=4, precision=0, form=form, n_steps=Nt, time_block=b, state_seed=2)
        C = np.zeros((4, E.size, Nt + 1), np.complex128)
        sigma = np.zeros((4, E.size))
        capi.tbpm_conductivity(ctx, lat, req, 0, E, C, sigma)
        out[form] = (C, sigma)
    C2 = np.zeros_like(out[1][0])
    s2 = np.zeros_like(out[1][1])
    capi.tbpm_conductivity(ctx, lat, capi.request(n_states=4, precision=0, form=1, n_steps=Nt, state_seed=2),
                           0, E, C2, s2)
    assert np.array_equal(C2, out[1][0]) and np.array_equal(s2, out[1][1])
    ref = out[0][0]
    scale = np.max(np.abs(ref), axis=2, keepdims=True)
    for form in (2, 1):
        assert np.max(np.abs(out[form][0] - ref) / scale) < 1e-4, form
    capi.tbpm_lattice_destroy(lat)


def test_conductivity_rejects_bad_direction_and_form(capi, ctx):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (8, 8), t=-2.7, seed=1))
    E = np.array([0.5])
    C = np.zeros((1, 1, 5), np.complex128)
    sigma = np.zeros((1, 1))
    with pytest.raises(capi.TbpmError):
        capi.tbpm_conductivity(ctx, lat, capi.request(n_states=1, n_steps=4), 2, E, C, sigma)
    with pytest.raises(capi.TbpmError):
        capi.tbpm_conductivity(ctx, lat, capi.request(n_states=1, n_steps=4, form=3), 0, E, C, sigma)
    capi.tbpm_lattice_destroy(lat)
