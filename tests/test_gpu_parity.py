"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Bars: bit-exact for lattice indexing, disorder, vacancy compaction, Philox draws and the
stencil/ELL neighbour sums; max_n |mu_gpu - mu_oracle| / |mu_0| <= 1e-5 for complex64 states
with FP64 reductions and <= 1e-11 for complex128; the same norms for C(t) (relative to C(0))
and for the DOS (relative to max D).
"""
import math

import numpy as np
import pytest

from oracle import lattice as olat, propagate as oprop, spectra as ospec, bessel as obes

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-11}  # C64, C128


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


def make(capi, ctx, kind, L, t=1.0, W=0.0, vac=0.0, seed=0x7B1A5, pbc=(1, 1, 1), path=0):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(kind, L, t=t, W=W, vacancy_frac=vac, seed=seed,
                                                          pbc=pbc, path=path))
    ol = olat.build_lattice(kind, tuple(L) + (1,) * (3 - len(L)), t=t, W=W, vacancy_frac=vac, seed=seed, pbc=pbc)
    return lat, ol


LATTICES = [
    ("square7x5_W1", dict(kind=0, L=(7, 5), t=1.0, W=1.0)),
    ("square9x4_open", dict(kind=0, L=(9, 4), t=-1.0, W=0.5, pbc=(0, 1, 1))),
    ("honey6x5_openx", dict(kind=1, L=(6, 5), t=-2.7, W=1.0, pbc=(0, 1, 1))),
    ("honey13x7", dict(kind=1, L=(13, 7), t=-2.7, W=2.0)),
    ("cubic3x4x5", dict(kind=2, L=(3, 4, 5), t=1.0, W=2.0)),
    ("cubic4x3x2_openz", dict(kind=2, L=(4, 3, 2), t=1.0, W=0.3, pbc=(1, 1, 0))),
    ("honey33x17_vac", dict(kind=1, L=(33, 17), t=-2.7, W=2.0, vac=0.05)),
    ("square20x20_vac", dict(kind=0, L=(20, 20), t=1.0, W=1.0, vac=0.1)),
    ("honey8x8_csr", dict(kind=1, L=(8, 8), t=-2.7, W=1.0, path=2)),
]


@pytest.mark.parametrize("name,spec", LATTICES, ids=[n for n, _ in LATTICES])
def test_lattice_bit_exact(capi, ctx, name, spec):
    lat, ol = make(capi, ctx, **spec)
    info = capi.tbpm_lattice_info(lat)
    assert info.n_sites == ol.n and info.n_full == ol.n_full
    assert (info.E_min, info.E_max, info.H0, info.half_width) == (ol.E_min, ol.E_max, ol.H0, ol.half_width)
    assert info.n_bonds == ol.H.nnz - np.count_nonzero(ol.H.diagonal()) or info.n_bonds == int(ol.degree.sum())
    z = info.coordination
    compact = np.zeros(ol.n_full, np.int64)
    V = np.zeros(ol.n)
    nbr = np.zeros((ol.n, z), np.int32)
    capi.tbpm_lattice_export(lat, compact, V, nbr)
    assert np.array_equal(compact, ol.compact)
    assert np.array_equal(V, ol.V)
    full_idx = np.flatnonzero(ol.active)
    want = ol.nbr_full[full_idx]
    want = np.where(want >= 0, ol.compact[np.maximum(want, 0)], -1)
    assert np.array_equal(nbr, want)
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("name,spec", LATTICES, ids=[n for n, _ in LATTICES])
@pytest.mark.parametrize("prec,S", [(0, 1), (0, 2), (0, 8), (1, 1), (1, 4)])
def test_stencil_neighbour_sums_exact(capi, ctx, name, spec, prec, S):
    """y = A x for integer-valued x through the hot-path kernel equals the oracle's adjacency."""
    lat, ol = make(capi, ctx, **spec)
    n = ol.n
    A = (ol.H - olat.sp.diags(ol.H.diagonal())).tocsr()
    A.data = np.round(A.data / ol.t)
    x = (np.arange(n)[:, None] + 1000.0 * np.arange(S)[None, :]) + 1j * (7.0 * np.arange(S)[None, :] + 1)
    y_ref = A @ x
    dt = np.complex64 if prec == 0 else np.complex128
    xs = np.ascontiguousarray(x.astype(dt))
    ys = np.zeros_like(xs)
    capi.tbpm_apply_hopping(ctx, lat, prec, S, xs, ys)
    assert np.array_equal(ys.astype(np.complex128), y_ref)
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("prec", [0, 1])
def test_random_states_match_oracle(capi, ctx, prec):
    lat, ol = make(capi, ctx, kind=1, L=(21, 9), t=-2.7, W=1.0, vac=0.07)
    S = 5
    req = capi.request(n_states=S, precision=prec, state_seed=0xABCDEF12345)
    dt = np.complex64 if prec == 0 else np.complex128
    out = np.zeros((S, ol.n), dt)
    draws = np.zeros((S, ol.n), np.uint32)
    capi.tbpm_states_export(ctx, lat, req, out, draws)
    from oracle.philox import draw_u32
    full_idx = np.flatnonzero(ol.active).astype(np.uint64)
    for s in range(S):
        assert np.array_equal(draws[s], draw_u32(0xABCDEF12345, full_idx, 2, s))
    ref = oprop.random_phase_states(ol, 0xABCDEF12345, S)
    if prec == 0:
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(out.real - ref.real) <= ulp) and np.all(np.abs(out.imag - ref.imag) <= ulp)
    else:
        assert np.max(np.abs(out - ref)) < 4e-16 / math.sqrt(ol.n) * 4
    capi.tbpm_lattice_destroy(lat)


def gpu_moments(capi, ctx, lat, S, M, prec, seed=3, sites=None):
    req = capi.request(n_states=S, precision=prec, n_moments=M, state_seed=seed, sites=sites)
    mu = np.zeros((req.n_states, M, 2))
    capi.tbpm_moments(ctx, lat, req, mu)
    return mu[..., 0] + 1j * mu[..., 1]


MOMENT_CASES = [
    ("honey20x12_c128", dict(kind=1, L=(20, 12), t=-2.7, W=1.0), 3, 512, 1),
    ("square64x64_c128", dict(kind=0, L=(64, 64), t=1.0, W=1.0), 1, 1024, 1),
    ("honey96x40_c64_S8", dict(kind=1, L=(96, 40), t=-2.7, W=0.0), 8, 1024, 0),
    ("honey70x33_c64_S5", dict(kind=1, L=(70, 33), t=-2.7, W=1.0), 5, 512, 0),
    ("square130x7_c64_S1", dict(kind=0, L=(130, 7), t=1.0, W=1.0), 1, 512, 0),
    ("cubic11x6x5_c64_S2", dict(kind=2, L=(11, 6, 5), t=1.0, W=2.0), 2, 256, 0),
    ("honey50x40_vac_c64", dict(kind=1, L=(50, 40), t=-2.7, W=2.0, vac=0.01), 4, 512, 0),
    ("honey30x20_vac_c128", dict(kind=1, L=(30, 20), t=-2.7, W=2.0, vac=0.03), 2, 400, 1),
]


@pytest.mark.parametrize("name,spec,S,M,prec", MOMENT_CASES, ids=[c[0] for c in MOMENT_CASES])
def test_moments_match_oracle(capi, ctx, name, spec, S, M, prec):
    lat, ol = make(capi, ctx, **spec)
    mu = gpu_moments(capi, ctx, lat, S, M, prec)
    psi = oprop.random_phase_states(ol, 3, S)
    for s in range(S):
        ref = oprop.moments(ol, psi[s], psi[s], M)
        err = np.max(np.abs(mu[s] - ref)) / abs(ref[0])
        assert err <= TOL[prec], (s, err)
    capi.tbpm_lattice_destroy(lat)


def test_ldos_site_states(capi, ctx):
    lat, ol = make(capi, ctx, kind=1, L=(17, 11), t=-2.7, W=1.0)
    sites = np.array([0, 5, 100, 373], np.int64)
    for prec in (0, 1):
        mu = gpu_moments(capi, ctx, lat, 4, 300, prec, sites=sites)
        st = oprop.site_states(ol, sites)
        for s in range(4):
            ref = oprop.moments(ol, st[s], st[s], 300)
            assert np.max(np.abs(mu[s] - ref)) <= TOL[prec]
    capi.tbpm_lattice_destroy(lat)


def test_stencil_and_csr_paths_agree(capi, ctx):
    spec = dict(kind=1, L=(40, 24), t=-2.7, W=1.0)
    a, _ = make(capi, ctx, **spec)
    b, _ = make(capi, ctx, path=2, **spec)
    assert capi.tbpm_lattice_info(b).path == 2
    ma = gpu_moments(capi, ctx, a, 4, 512, 1)
    mb = gpu_moments(capi, ctx, b, 4, 512, 1)
    assert np.max(np.abs(ma - mb)) < 1e-12
    capi.tbpm_lattice_destroy(a)
    capi.tbpm_lattice_destroy(b)


def test_moments_deterministic(capi, ctx):
    lat, _ = make(capi, ctx, kind=1, L=(256, 64), t=-2.7, W=1.0)
    m1 = gpu_moments(capi, ctx, lat, 8, 256, 0)
    m2 = gpu_moments(capi, ctx, lat, 8, 256, 0)
    assert np.array_equal(m1, m2)
    capi.tbpm_lattice_destroy(lat)


def gpu_corr(capi, ctx, lat, S, Nt, prec, form, b=0, seed=3):
    req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=seed)
    C = np.zeros((S, Nt + 1, 2))
    capi.tbpm_correlation(ctx, lat, req, C)
    return C[..., 0] + 1j * C[..., 1]


@pytest.mark.parametrize("prec", [1, 0])
def test_correlation_forms_match_oracle(capi, ctx, prec):
    """Sequential, moment-based and state-based forms (Sec. II.A) against the oracle's
    sequential propagation on the 16x16 square lattice with W = 1."""
    lat, ol = make(capi, ctx, kind=0, L=(16, 16), t=1.0, W=1.0)
    Nt, S = 40, 2
    psi = oprop.random_phase_states(ol, 3, S)
    refs = [oprop.correlation_sequential(ol, psi[s], Nt) for s in range(S)]
    for form, b in ((capi.SEQUENTIAL, 0), (capi.CONCURRENT_M, 0), (capi.CONCURRENT_S, 7),
                    (capi.CONCURRENT_S, 40), (capi.CONCURRENT_S, 0)):
        C = gpu_corr(capi, ctx, lat, S, Nt, prec, form, b)
        for s in range(S):
            err = np.max(np.abs(C[s] - refs[s])) / abs(refs[s][0])
            assert err <= TOL[prec], (form, b, s, err)
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("pbc", [(1, 1, 1), (0, 1, 1)])
def test_correlation_forms_through_window_sweep(capi, ctx, pbc):
    """Honeycomb lattices wide enough for the register sweep's window pass (four Chebyshev terms
    of a time block per pass into four buffer slots): the sequential form (b = 1) and the time
    blocks of every size against the oracle's sequential propagation, periodic and open in x."""
    lat, ol = make(capi, ctx, kind=1, L=(100, 64), t=-2.7, W=1.0, pbc=pbc)
    Nt, S = 30, 4
    psi = oprop.random_phase_states(ol, 3, S)
    refs = {s: oprop.correlation_sequential(ol, psi[s], Nt) for s in (0, S - 1)}
    for form, b in ((capi.SEQUENTIAL, 0), (capi.CONCURRENT_S, 7), (capi.CONCURRENT_S, 30), (capi.CONCURRENT_S, 0),
                    (capi.CONCURRENT_M, 0)):
        C = gpu_corr(capi, ctx, lat, S, Nt, 0, form, b)
        for s, ref in refs.items():
            err = np.max(np.abs(C[s] - ref)) / abs(ref[0])
            assert err <= TOL[0], (form, b, s, err)
    capi.tbpm_lattice_destroy(lat)


def test_correlation_vacancy_lattice(capi, ctx):
    lat, ol = make(capi, ctx, kind=1, L=(24, 16), t=-2.7, W=2.0, vac=0.02)
    psi = oprop.random_phase_states(ol, 3, 1)[0]
    ref = oprop.correlation_sequential(ol, psi, 25)
    for form, b in ((capi.SEQUENTIAL, 0), (capi.CONCURRENT_M, 0), (capi.CONCURRENT_S, 6)):
        C = gpu_corr(capi, ctx, lat, 1, 25, 1, form, b)
        assert np.max(np.abs(C[0] - ref)) <= 1e-11
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("prec", [1, 0])
def test_jackson_dos_matches_oracle(capi, ctx, prec):
    lat, ol = make(capi, ctx, kind=1, L=(32, 24), t=-2.7, W=1.0)
    S, M, nE = 3, 512, 301
    E = np.linspace(ol.H0 - 1.02 * ol.half_width, ol.H0 + 1.02 * ol.half_width, nE)
    req = capi.request(n_states=S, precision=prec, n_moments=M, dos_method=capi.DOS_JACKSON)
    D = np.zeros((S, nE))
    capi.tbpm_dos(ctx, lat, req, E, D)
    psi = oprop.random_phase_states(ol, 1, S)
    for s in range(S):
        mu = oprop.moments(ol, psi[s], psi[s], M)
        ref = ospec.dos_jackson(mu, E, ol.H0, ol.half_width)
        assert np.max(np.abs(D[s] - ref)) / np.max(ref) <= TOL[prec]
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_fourier_dos_matches_oracle(capi, ctx, form):
    lat, ol = make(capi, ctx, kind=0, L=(16, 16), t=1.0, W=1.0)
    Nt, nE = 60, 200
    E = np.linspace(ol.H0 - ol.half_width, ol.H0 + ol.half_width, nE)
    req = capi.request(n_states=1, precision=1, form=form, n_steps=Nt, time_block=9,
                       dos_method=capi.DOS_FOURIER, window=capi.WINDOW_HANN)
    D = np.zeros((1, nE))
    capi.tbpm_dos(ctx, lat, req, E, D)
    psi = oprop.random_phase_states(ol, 1, 1)[0]
    C = oprop.correlation_sequential(ol, psi, Nt)
    ref = ospec.dos_fourier(C, math.pi / ol.half_width, E, ospec.WINDOW_HANN)
    assert np.max(np.abs(D[0] - ref)) / np.max(np.abs(ref)) <= 1e-11
    capi.tbpm_lattice_destroy(lat)


# ---------------------------------------------------------------- edge cases

def test_edge_sizes(capi, ctx):
    # one-cell-wide periodic lattices: bonds wrap onto the same site and add up
    for spec in (dict(kind=0, L=(1, 9), W=1.0), dict(kind=1, L=(1, 1), W=1.0), dict(kind=0, L=(2, 2), W=1.0),
                 dict(kind=2, L=(1, 1, 3), W=0.5)):
        lat, ol = make(capi, ctx, **spec)
        mu = gpu_moments(capi, ctx, lat, 1, 64, 1)
        psi = oprop.random_phase_states(ol, 3, 1)[0]
        assert np.max(np.abs(mu[0] - oprop.moments(ol, psi, psi, 64))) <= 1e-11
        capi.tbpm_lattice_destroy(lat)


def test_minimal_moments_and_max_states(capi, ctx):
    lat, ol = make(capi, ctx, kind=1, L=(10, 10), t=-2.7, W=1.0)
    mu = gpu_moments(capi, ctx, lat, 32, 2, 0)
    psi = oprop.random_phase_states(ol, 3, 32)
    for s in (0, 17, 31):
        ref = oprop.moments(ol, psi[s], psi[s], 2)
        assert np.max(np.abs(mu[s] - ref)) <= 1e-6
    capi.tbpm_lattice_destroy(lat)


def test_invalid_requests_raise(capi, ctx):
    lat, _ = make(capi, ctx, kind=0, L=(8, 8))
    mu = np.zeros((1, 8, 2))
    for kw in (dict(n_moments=7), dict(n_moments=0), dict(n_states=0), dict(n_states=33)):
        args = dict(n_states=1, n_moments=8)
        args.update(kw)
        with pytest.raises(capi.TbpmError):
            capi.tbpm_moments(ctx, lat, capi.request(**args), np.zeros((max(1, args["n_states"]), 8, 2)))
    with pytest.raises(capi.TbpmError):
        capi.tbpm_moments(ctx, lat, capi.request(sites=[64], n_moments=8), mu)
    for d in (dict(kind=5, L=(4, 4)), dict(kind=0, L=(0, 4)), dict(kind=0, L=(4, 4), t=0.0),
              dict(kind=0, L=(4, 4), vacancy_frac=1.0), dict(kind=0, L=(4, 4), W=-1.0)):
        with pytest.raises(capi.TbpmError):
            capi.tbpm_lattice_create(ctx, capi.lattice_desc(**d))
    capi.tbpm_lattice_destroy(lat)


# ---------------------------------------------------------------- full benchmark size, sampled

def test_full_size_graphene_sampled(capi, ctx):
    """Honeycomb 2048x2048 (8,388,608 sites), 8 states, 4096 moments in the benchmark's
    launch configuration: the first 32 moments of state 0 against the oracle, and
    invariants of all 4096 x 8 (mu_0 = 1, |mu_n| <= 1, odd moments ~ 0 by bipartite symmetry
    of the clean lattice only in expectation, so only bounded)."""
    lat, ol = make(capi, ctx, kind=1, L=(2048, 2048), t=-2.7, W=0.0)
    S, M = 8, 4096
    mu = gpu_moments(capi, ctx, lat, S, M, 0, seed=1)
    assert np.max(np.abs(mu[:, 0] - 1.0)) < 1e-6
    assert np.max(np.abs(mu)) <= 1.0 + 1e-6
    psi = oprop.random_phase_states(ol, 1, 1)[0]
    ref = oprop.moments(ol, psi, psi, 32)
    assert np.max(np.abs(mu[0, :32] - ref)) <= 1e-5
    capi.tbpm_lattice_destroy(lat)


# ---------------------------------------------------------------- temporal fusion (2 or 4 steps per pass)

FUSED_CASES = [
    ("honey48x32_exact_tile", dict(kind=1, L=(48, 32), t=-2.7, W=0.0), 2, 64),
    ("honey88x56_two_tiles", dict(kind=1, L=(88, 56), t=-2.7, W=0.0), 2, 66),
    ("honey101x77_ragged_W1", dict(kind=1, L=(101, 77), t=-2.7, W=1.0), 8, 202),
    ("honey90x70_open_x", dict(kind=1, L=(90, 70), t=-2.7, W=0.5, pbc=(0, 1, 1)), 4, 130),
    ("honey60x100_open_y", dict(kind=1, L=(60, 100), t=1.0, W=2.0, pbc=(1, 0, 1)), 16, 96),
    ("honey50x40_open_xy_S32", dict(kind=1, L=(50, 40), t=-2.7, W=1.0, pbc=(0, 0, 1)), 32, 38),
    ("honey300x150_three_segments", dict(kind=1, L=(300, 150), t=-2.7, W=0.7), 8, 40),
]


@pytest.mark.parametrize("mode", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("name,spec,S,M", FUSED_CASES, ids=[c[0] for c in FUSED_CASES])
def test_fused_passes_match_unfused_and_oracle(capi, ctx, name, spec, S, M, mode):
    lat, ol = make(capi, ctx, **spec)
    capi.tbpm_set_fusion(ctx, mode)
    mf = gpu_moments(capi, ctx, lat, S, M, 0)
    capi.tbpm_set_fusion(ctx, 0)
    mu = gpu_moments(capi, ctx, lat, S, M, 0)
    capi.tbpm_set_fusion(ctx, 8)
    assert np.max(np.abs(mf - mu)) <= 1e-6
    psi = oprop.random_phase_states(ol, 3, S)
    for s in (0, S - 1):
        ref = oprop.moments(ol, psi[s], psi[s], M)
        assert np.max(np.abs(mf[s] - ref)) <= 1e-5
    capi.tbpm_lattice_destroy(lat)


def test_fusion_autotune_picks_a_timed_mode_and_matches(capi, ctx):
    """Mode -1 times modes 0, 4, 5, 8 on the request's lattice shape and uses the fastest; the
    moments agree with the one-step pass within the complex64 tolerance."""
    lat, ol = make(capi, ctx, kind=1, L=(256, 200), t=-2.7, W=0.5)
    capi.tbpm_set_fusion(ctx, -1)
    ma = gpu_moments(capi, ctx, lat, 8, 160, 0)
    rep = capi.tbpm_fusion_report(ctx)
    capi.tbpm_set_fusion(ctx, 0)
    m0 = gpu_moments(capi, ctx, lat, 8, 160, 0)
    capi.tbpm_set_fusion(ctx, 8)
    assert set(rep) == {0, 4, 5, 8} and all(v > 0 for v in rep.values())
    assert np.max(np.abs(ma - m0)) <= 1e-6
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("spec,S,prec", [(dict(kind=1, L=(96, 64), t=-2.7, W=0.5), 8, 0),
                                         (dict(kind=0, L=(64, 64), t=1.0, W=1.0), 1, 1)])
def test_graph_replay_is_bit_identical(capi, ctx, spec, S, prec):
    """The second identical moment request is captured into a CUDA graph, the third replays it;
    all equal the eager result bit for bit, and replays count their kernels."""
    lat, _ = make(capi, ctx, **spec)
    capi.tbpm_set_graphs(ctx, False)
    ref = gpu_moments(capi, ctx, lat, S, 256, prec)
    capi.tbpm_set_graphs(ctx, True)
    outs = []
    for _ in range(3):
        c0 = capi.tbpm_launch_count(ctx)
        outs.append(gpu_moments(capi, ctx, lat, S, 256, prec))
        assert capi.tbpm_launch_count(ctx) - c0 >= 2
    for o in outs:
        assert np.array_equal(o, ref)
    capi.tbpm_lattice_destroy(lat)


# ---------------------------------------------------------------- headline moment counts, every moment

_ORACLE_CACHE = {}


def oracle_moments_cached(key, ol, seed, s, M):
    """Oracle moments of state s (plain definition), kept across the fusion modes of one case."""
    k = (key, seed, s, M)
    if k not in _ORACLE_CACHE:
        psi = oprop.random_phase_states(ol, seed, s + 1)[s]
        _ORACLE_CACHE[k] = oprop.moments(ol, psi, psi, M)
    return _ORACLE_CACHE[k]


HEADLINE_CASES = [
    # the benchmark's state block and moment count on a lattice wide and tall enough for many
    # bands and row segments of the fused sweep (2047 fused steps)
    ("honey512x384_S8_M4096", dict(kind=1, L=(512, 384), t=-2.7, W=0.0), 8, 4096, (0, 7)),
    # the 1e9-site workload's state block, moment count and disorder (4095 steps)
    ("honey200x150_W1_S4_M8192", dict(kind=1, L=(200, 150), t=-2.7, W=1.0), 4, 8192, (0, 3)),
]


@pytest.mark.parametrize("mode", [0, 5, 8])
@pytest.mark.parametrize("name,spec,S,M,check", HEADLINE_CASES, ids=[c[0] for c in HEADLINE_CASES])
def test_headline_moment_counts_match_oracle(capi, ctx, name, spec, S, M, check, mode):
    """Every one of the M moments of two states at the benchmark's M = 4096 (S = 8) and the
    1e9-site workload's M = 8192 (S = 4), complex64 states with FP64 reductions, through the
    one-step pass (mode 0) and the four-step fused passes (mode 5: shared-memory level rings,
    mode 8: register-resident sweep with TMA row copies): max_n |dmu_n| / |mu_0| <= 1e-5 against
    the oracle's plain FP64 moments."""
    lat, ol = make(capi, ctx, **spec)
    capi.tbpm_set_fusion(ctx, mode)
    try:
        mu = gpu_moments(capi, ctx, lat, S, M, 0, seed=2)
    finally:
        capi.tbpm_set_fusion(ctx, 8)
    capi.tbpm_lattice_destroy(lat)
    for s in check:
        ref = oracle_moments_cached(name, ol, 2, s, M)
        err = np.max(np.abs(mu[s] - ref)) / abs(ref[0])
        assert err <= 1e-5, (s, err)


# ---------------------------------------------------------------- the 1.015e9-site lattice, sampled

def test_largest_lattice_sampled_sites_match_oracle_windows(capi, ctx):
    """Honeycomb 22528 x 22528 cells (1,015,021,568 sites), t = -2.7 eV, V in [-0.5, 0.5) eV: the
    largest workload, in the default fused pass with disorder, at byte offsets far beyond 2^32.
    Its Gershgorin bounds equal the oracle's (from the disorder range over all sites, stored by
    tests/golden/make_disorder_range.py), and the LDOS moments of four sites (a corner whose light
    cone wraps both periodic directions, the last site, the centre, a band edge of the sweep)
    equal those of the oracle on a window of the lattice around each site, exact while the
    moment index stays below the window's radius."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "honeycomb22528_W1_disorder_range.json")) as f:
        rng = json.load(f)
    Lx = Ly = 22528
    t, W, seed = -2.7, 1.0, 0x7B1A5
    assert rng["lattice"]["L"] == [Lx, Ly] and rng["lattice"]["W"] == W and rng["lattice"]["seed"] == seed
    E_min = rng["V_min"] - 3 * abs(t)
    E_max = rng["V_max"] + 3 * abs(t)
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (Lx, Ly), t=t, W=W, seed=seed))
    try:
        info = capi.tbpm_lattice_info(lat)
        assert info.n_sites == 2 * Lx * Ly
        assert (info.E_min, info.E_max) == (E_min, E_max)
        cells = [(0, 0, 0), (Lx - 1, Ly - 1, 1), (Lx // 2, Ly // 2 - 1, 0), (60 * 187, 7509, 1)]
        sites = np.array([2 * (y * Lx + x) + s for x, y, s in cells], np.int64)
        M = 256
        mu = gpu_moments(capi, ctx, lat, 4, M, 0, sites=sites)
    finally:
        capi.tbpm_lattice_destroy(lat)
    for k, (x, y, s) in enumerate(cells):
        wl, ia, ib, full = olat.honeycomb_window((Lx, Ly), (x, y), M, t, W, seed, E_min, E_max)
        local = ia if s == 0 else ib
        assert full[local] == sites[k]
        e = np.zeros(wl.n, np.complex128)
        e[local] = 1.0
        ref = oprop.moments(wl, e, e, M)
        assert np.max(np.abs(mu[k] - ref)) <= 1e-5, (k, np.max(np.abs(mu[k] - ref)))


def test_moment_pass_kind_names_the_kernel(capi, ctx):
    """tbpm_moment_pass_kind names the kernel family that carries a request's recurrence."""
    cases = [
        (dict(kind=1, L=(100, 64), t=-2.7), dict(n_states=8, n_moments=256), 8, capi.PASS_SWEEP),
        (dict(kind=1, L=(100, 64), t=-2.7), dict(n_states=8, n_moments=256), 5, capi.PASS_ROWS),
        (dict(kind=1, L=(100, 64), t=-2.7), dict(n_states=8, n_moments=256), 1, capi.PASS_TILES),
        (dict(kind=1, L=(100, 64), t=-2.7), dict(n_states=8, n_moments=256), 0, capi.PASS_STENCIL),
        (dict(kind=1, L=(100, 64), t=-2.7), dict(n_states=1, n_moments=256), 8, capi.PASS_STENCIL),
        (dict(kind=1, L=(100, 64), t=-2.7), dict(n_states=8, n_moments=256, precision=1), 8, capi.PASS_STENCIL),
        (dict(kind=1, L=(40, 40), t=-2.7), dict(n_states=8, n_moments=256), 8, capi.PASS_STENCIL),
        (dict(kind=0, L=(64, 64), t=1.0), dict(n_states=8, n_moments=256), 8, capi.PASS_STENCIL),
        (dict(kind=1, L=(40, 40), t=-2.7, vac=0.05), dict(n_states=2, n_moments=64), 8, capi.PASS_ELL),
    ]
    for spec, rk, mode, want in cases:
        lat, _ = make(capi, ctx, **spec)
        capi.tbpm_set_fusion(ctx, mode)
        try:
            assert capi.tbpm_moment_pass_kind(ctx, lat, capi.request(**rk)) == want, (spec, rk, mode)
        finally:
            capi.tbpm_set_fusion(ctx, 8)
            capi.tbpm_lattice_destroy(lat)
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (70, 36), t=-2.7, cutoff=7.1, decay=0.3187))
    assert capi.tbpm_moment_pass_kind(ctx, lat, capi.request(n_states=2, n_moments=64)) == capi.PASS_TAPS
    capi.tbpm_lattice_destroy(lat)
