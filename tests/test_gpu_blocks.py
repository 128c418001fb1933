"""Buffered time blocks (Sec. II.B, Eq. TE): the recurrence writes phi_n into buffer slots and one
flush per 32 terms adds sum_n c_n(j tau~) phi_n to every accumulator of the block.  Against the
FP64 oracle and against the unbuffered accumulation (one accumulator update per term) on the
stencil, ELL and tap paths, in complex64 and complex128."""
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
    capi.tbpm_set_block_buffering(h, True)
    capi.tbpm_destroy(h)


SPECS = [
    ("honey24x16_stencil", dict(kind=1, L=(24, 16), t=-2.7, W=1.0, seed=3)),
    ("square20x18_vac_ell", dict(kind=0, L=(20, 18), t=1.0, W=1.0, vacancy_frac=0.05, seed=4)),
    ("honey70x20_taps", dict(kind=1, L=(70, 20), t=-2.7, W=0.5, seed=5, cutoff=3.1, decay=0.3187)),
]


def _oracle(spec):
    L = tuple(spec["L"]) + (1,) * (3 - len(spec["L"]))
    return olat.build_lattice(spec["kind"], L, t=spec["t"], W=spec["W"], vacancy_frac=spec.get("vacancy_frac", 0.0),
                              seed=spec["seed"], cutoff=spec.get("cutoff", 0.0), decay=spec.get("decay", 0.0))


def _corr(capi, ctx, lat, S, Nt, prec, form, b):
    req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=3)
    C = np.zeros((S, Nt + 1, 2))
    capi.tbpm_correlation(ctx, lat, req, C)
    return C[..., 0] + 1j * C[..., 1]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,spec", SPECS, ids=[n for n, _ in SPECS])
def test_buffered_blocks_match_oracle_and_unbuffered(capi, ctx, name, spec, prec):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle(spec)
    S, Nt = 2, 45
    psi = oprop.random_phase_states(ol, 3, S)
    refs = [oprop.correlation_sequential(ol, psi[s], Nt) for s in range(S)]
    for form, b in ((capi.SEQUENTIAL, 0), (capi.CONCURRENT_S, 9), (capi.CONCURRENT_S, 45), (capi.CONCURRENT_S, 0)):
        capi.tbpm_set_block_buffering(ctx, True)
        Cb = _corr(capi, ctx, lat, S, Nt, prec, form, b)
        Cb2 = _corr(capi, ctx, lat, S, Nt, prec, form, b)
        capi.tbpm_set_block_buffering(ctx, False)
        Cu = _corr(capi, ctx, lat, S, Nt, prec, form, b)
        capi.tbpm_set_block_buffering(ctx, True)
        if b > 0 or form == capi.SEQUENTIAL:  # b = 0 is chosen from measured pass times per call
            assert np.array_equal(Cb, Cb2)
        else:
            assert np.max(np.abs(Cb - Cb2)) <= 2 * TOL[prec]
        for s in range(S):
            assert np.max(np.abs(Cb[s] - refs[s])) / abs(refs[s][0]) <= TOL[prec], (form, b, s)
            assert np.max(np.abs(Cb[s] - Cu[s])) / abs(refs[s][0]) <= 2 * TOL[prec], (form, b, s)
    capi.tbpm_lattice_destroy(lat)


def test_buffered_quasi_eigenstates_match_oracle(capi, ctx):
    spec = SPECS[0][1]
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(**spec))
    ol = _oracle(spec)
    E = np.array([-4.0, 0.3, 2.2])
    Nt, S = 37, 2
    out = np.zeros((E.size, S, ol.n), np.complex128)
    capi.tbpm_quasi_eigenstates(ctx, lat, capi.request(n_states=S, precision=1, form=capi.CONCURRENT_S, n_steps=Nt,
                                                       time_block=6, state_seed=8), E, out)
    psi = oprop.random_phase_states(ol, 8, S)
    for s in range(S):
        ref = oqe.qe_concurrent_e(ol, psi[s], E, Nt)
        for k in range(E.size):
            assert np.max(np.abs(out[k, s] - ref[k])) / np.max(np.abs(ref[k])) <= TOL[1]
    capi.tbpm_lattice_destroy(lat)
