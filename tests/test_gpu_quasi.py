"""Quasi-eigenstates on the GPU (Sec. IV) in the sequential, state-based and energy-based forms
against the FP64 oracle.  Norm: max |Psi_gpu - Psi_oracle| / max |Psi_oracle| per energy,
<= 1e-11 for complex128 and <= 1e-5 for complex64."""
import math

import numpy as np
import pytest

from oracle import lattice as olat, propagate as oprop, quasi as oqe

pytestmark = pytest.mark.gpu
TOL = {0: 1e-5, 1: 1e-11}


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


CASES = [
    ("honey12x10_W15", dict(kind=1, L=(12, 10), t=-2.7, W=1.5, seed=21), 2),
    ("square9x11_open", dict(kind=0, L=(9, 11), t=1.0, W=1.0, seed=22, pbc=(0, 1, 1)), 1),
    ("honey14x9_vac", dict(kind=1, L=(14, 9), t=-2.7, W=2.0, vacancy_frac=0.04, seed=23), 2),
]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("form,b", [(0, 0), (2, 5), (2, 0), (3, 0)])
@pytest.mark.parametrize("name,spec,S", CASES, ids=[c[0] for c in CASES])
def test_quasi_eigenstates_match_oracle(capi, ctx, name, spec, S, form, b, prec):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = olat.build_lattice(spec["kind"], tuple(spec["L"]) + (1,), t=spec["t"], W=spec["W"],
                            vacancy_frac=spec.get("vacancy_frac", 0.0), seed=spec["seed"],
                            pbc=spec.get("pbc", (1, 1, 1)))
    E = np.array([-5.0, -1.1, 0.0, 0.7, 4.2])
    Nt = 23
    req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=8)
    dt = np.complex64 if prec == 0 else np.complex128
    out = np.zeros((E.size, S, ol.n), dt)
    capi.tbpm_quasi_eigenstates(ctx, lat, req, E, out)
    psi = oprop.random_phase_states(ol, 8, S)
    for s in range(S):
        ref = oqe.qe_concurrent_e(ol, psi[s], E, Nt)
        for k in range(E.size):
            err = np.max(np.abs(out[k, s] - ref[k])) / np.max(np.abs(ref[k]))
            assert err <= TOL[prec], (form, b, s, k, err)
    capi.tbpm_lattice_destroy(lat)


def test_quasi_eigenstate_overlap_equals_fourier_dos(capi, ctx):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (30, 20), t=-2.7, W=1.0, seed=4))
    E = np.linspace(-8, 8, 7)
    Nt = 40
    req = capi.request(n_states=1, precision=1, form=3, n_steps=Nt, state_seed=3)
    qe = np.zeros((E.size, 1, 1200), np.complex128)
    capi.tbpm_quasi_eigenstates(ctx, lat, req, E, qe)
    st = np.zeros((1, 1200), np.complex128)
    capi.tbpm_states_export(ctx, lat, req, st)
    D = np.zeros((1, E.size))
    capi.tbpm_dos(ctx, lat, capi.request(n_states=1, precision=1, form=1, n_steps=Nt, state_seed=3,
                                         dos_method=capi.DOS_FOURIER), E, D)
    ov = np.array([np.vdot(st[0], qe[k, 0]) for k in range(E.size)])
    assert np.max(np.abs(ov - D[0])) < 1e-11
    capi.tbpm_lattice_destroy(lat)
