"""Long-range hopping lattices (all sites within a cutoff, t(r) = t exp(-(r-1)/decay); the
stand-in for the dense Hamiltonians of density D_H = 60..230 of Sec. IV) on the GPU against the
FP64 oracle: the Hamiltonian itself, moments, correlations in every form, the Jackson DOS,
quasi-eigenstates, the Fermi-Dirac operator, dynamical polarization and charge density, and the
calls that reject such lattices.

Bars as for the nearest-neighbour lattices: H to 1e-14 (FP64 weights), moments and C(t)
<= 1e-5 (complex64) / 1e-11 (complex128) relative to mu_0 / C(0); the response quantities at
the response tests' 3e-5 / 1e-10."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lattice as olat, propagate as oprop, spectra as ospec, quasi as oqe, response as R
from oracle import charge as ocd

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-11}
TOL_RESP = {0: 3e-5, 1: 1e-10}
DECAY = 0.3187


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


def make(capi, ctx, kind, L, t=-2.7, W=0.0, vac=0.0, seed=0x7B1A5, pbc=(1, 1, 1), cutoff=3.1, decay=DECAY):
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(kind, L, t=t, W=W, vacancy_frac=vac, seed=seed,
                                                          pbc=pbc, cutoff=cutoff, decay=decay))
    ol = olat.build_lattice(kind, tuple(L) + (1,) * (3 - len(L)), t=t, W=W, vacancy_frac=vac, seed=seed, pbc=pbc,
                            cutoff=cutoff, decay=decay)
    return lat, ol


LATTICES = [
    ("honey9x7_c5.1", dict(kind=1, L=(9, 7), W=1.0, cutoff=5.1)),
    ("honey12x10_c3.1_openx", dict(kind=1, L=(12, 10), W=0.5, pbc=(0, 1, 1), cutoff=3.1)),
    ("honey4x3_c4.1_images", dict(kind=1, L=(4, 3), W=1.0, cutoff=4.1)),
    ("honey14x9_c2.1_vac", dict(kind=1, L=(14, 9), W=2.0, vac=0.05, cutoff=2.1)),
    ("square11x9_c2.9", dict(kind=0, L=(11, 9), t=1.0, W=1.0, cutoff=2.9, decay=0.6)),
    ("cubic5x4x6_c1.8_openz", dict(kind=2, L=(5, 4, 6), t=1.0, W=1.0, pbc=(1, 1, 0), cutoff=1.8, decay=0.5)),
]


@pytest.mark.parametrize("name,spec", LATTICES, ids=[n for n, _ in LATTICES])
def test_hamiltonian_matches_oracle(capi, ctx, name, spec):
    """H rebuilt from the exported ELL lists, tap hoppings and V equals the oracle's H; bounds,
    site counts and bond counts agree."""
    lat, ol = make(capi, ctx, **spec)
    info = capi.tbpm_lattice_info(lat)
    assert info.n_sites == ol.n and info.path == 2
    assert info.n_bonds == int(np.asarray(ol.degree).sum())
    z = info.coordination
    off, tk = capi.tbpm_lattice_taps(lat)
    nbr = np.zeros(ol.n * z, np.int32)
    V = np.zeros(ol.n)
    capi.tbpm_lattice_export(lat, None, V, nbr)
    nbr = nbr.reshape(ol.n, z)
    rows = np.repeat(np.arange(ol.n), z)
    cols = nbr.ravel()
    keep = cols >= 0
    Hg = sp.coo_matrix((np.tile(tk, ol.n)[keep], (rows[keep], cols[keep])), shape=(ol.n, ol.n)).tocsr()
    Hg = Hg + sp.diags(V)
    assert abs(Hg - ol.H).max() < 1e-14 * abs(spec.get("t", -2.7)) * 10
    assert abs(info.E_max - ol.E_max) < 1e-13 and abs(info.E_min - ol.E_min) < 1e-13
    assert abs(info.half_width - ol.half_width) < 1e-13
    capi.tbpm_lattice_destroy(lat)


def test_taps_of_the_benchmark_densities(capi, ctx):
    """Cutoffs 5.1, 7.1 and 9.7 give D_H = 61, 124 and 235 (taps + diagonal); tap hoppings follow
    t(r) with r from the tap offsets."""
    for cutoff, dh in ((5.1, 61), (7.1, 124), (9.7, 235)):
        lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (24, 24), t=-2.7, cutoff=cutoff, decay=DECAY))
        info = capi.tbpm_lattice_info(lat)
        assert info.coordination + 1 == dh
        off, tk = capi.tbpm_lattice_taps(lat)
        r = np.linalg.norm(off[:, 0:1] * np.array([1.5, math.sqrt(3) / 2]) +
                           off[:, 1:2] * np.array([1.5, -math.sqrt(3) / 2]) + off[:, 3:4] * np.array([1.0, 0.0]),
                           axis=1)
        assert np.all((r > 0.99) & (r <= cutoff))
        assert np.max(np.abs(tk - (-2.7) * np.exp(-(r - 1) / DECAY))) < 1e-14
        capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("name,spec", LATTICES[:4], ids=[n for n, _ in LATTICES[:4]])
@pytest.mark.parametrize("prec,S", [(0, 2), (0, 8), (1, 1)])
def test_hopping_apply_matches_oracle(capi, ctx, name, spec, prec, S):
    """y = sum_j (H_ij / t) x_j (off-diagonal) through the hot-path kernel."""
    lat, ol = make(capi, ctx, **spec)
    n = ol.n
    A = (ol.H - sp.diags(ol.H.diagonal())).tocsr() / ol.t
    # images landing on the site itself sit on the diagonal of H; add them back
    off, tk = capi.tbpm_lattice_taps(lat)
    nbr = np.zeros(n * len(tk), np.int32)
    capi.tbpm_lattice_export(lat, None, None, nbr)
    nbr = nbr.reshape(n, len(tk))
    selfw = np.array([np.sum(tk[nbr[i] == i]) for i in range(n)]) / ol.t
    A = A + sp.diags(selfw)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((n, S)) + 1j * rng.standard_normal((n, S))
    dt = np.complex64 if prec == 0 else np.complex128
    xs = np.ascontiguousarray(x.astype(dt))
    ys = np.zeros_like(xs)
    capi.tbpm_apply_hopping(ctx, lat, prec, S, xs, ys)
    ref = A @ xs.astype(np.complex128)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(ys - ref)) / scale <= (2e-6 if prec == 0 else 1e-14)
    capi.tbpm_lattice_destroy(lat)


def gpu_moments(capi, ctx, lat, S, M, prec, seed=3):
    req = capi.request(n_states=S, precision=prec, n_moments=M, state_seed=seed)
    mu = np.zeros((S, M, 2))
    capi.tbpm_moments(ctx, lat, req, mu)
    return mu[..., 0] + 1j * mu[..., 1]


MOMENT_CASES = [
    ("honey20x16_c5.1_c128", dict(kind=1, L=(20, 16), W=1.0, cutoff=5.1), 2, 400, 1),
    ("honey24x24_c9.7_c64_S8", dict(kind=1, L=(24, 24), W=0.5, cutoff=9.7), 8, 256, 0),
    ("honey30x18_c7.1_vac_c64", dict(kind=1, L=(30, 18), W=1.0, vac=0.02, cutoff=7.1), 4, 300, 0),
    ("square40x30_c3.3_c64_S1", dict(kind=0, L=(40, 30), t=1.0, W=1.0, cutoff=3.3, decay=0.7), 1, 512, 0),
    ("cubic8x7x6_c2.3_c128", dict(kind=2, L=(8, 7, 6), t=1.0, W=1.0, cutoff=2.3, decay=0.5), 3, 256, 1),
    # matrix-free tap kernel (clean or disordered, no vacancies, complex64, >= 2 states)
    # (tiles of 64 honeycomb / 128 square cells by 16 rows: every case spans several tiles with
    # ragged tails, or is smaller than one tile)
    ("taps_honey66x18_c9.7_S2", dict(kind=1, L=(66, 18), W=0.0, cutoff=9.7), 2, 512, 0),
    ("taps_honey70x33_c5.1_open_S4", dict(kind=1, L=(70, 33), W=1.0, pbc=(0, 1, 1), cutoff=5.1), 4, 300, 0),
    ("taps_honey5x4_c4.1_images_S3", dict(kind=1, L=(5, 4), W=1.0, cutoff=4.1), 3, 256, 0),
    ("taps_square130x17_c3.3_openy_S2", dict(kind=0, L=(130, 17), t=1.0, W=0.5, pbc=(1, 0, 1), cutoff=3.3,
                                         decay=0.7), 2, 400, 0),
    ("taps_honey66x20_c7.1_S16", dict(kind=1, L=(66, 20), W=0.3, cutoff=7.1), 16, 128, 0),
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


def test_tap_kernel_agrees_with_ell_lists(capi, ctx):
    """The matrix-free tap kernel (path AUTO) and the ELL lists (path CSR) give the same moments
    to FP32 rounding on the benchmark's densest cutoff; both are deterministic."""
    a = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (96, 64), t=-2.7, W=0.5, seed=0x7B1A5, cutoff=9.7,
                                                        decay=DECAY))
    b = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (96, 64), t=-2.7, W=0.5, seed=0x7B1A5, cutoff=9.7,
                                                        decay=DECAY, path=2))
    ma = gpu_moments(capi, ctx, a, 8, 512, 0)
    mb = gpu_moments(capi, ctx, b, 8, 512, 0)
    assert not np.array_equal(ma, mb)          # two different kernels ran
    assert np.max(np.abs(ma - mb)) < 1e-5
    assert np.array_equal(ma, gpu_moments(capi, ctx, a, 8, 512, 0))
    capi.tbpm_lattice_destroy(a)
    capi.tbpm_lattice_destroy(b)


@pytest.mark.parametrize("prec", [1, 0])
def test_correlation_forms_match_oracle(capi, ctx, prec):
    lat, ol = make(capi, ctx, kind=1, L=(14, 12), W=1.0, cutoff=5.1)
    Nt, S = 30, 2
    psi = oprop.random_phase_states(ol, 3, S)
    refs = [oprop.correlation_sequential(ol, psi[s], Nt) for s in range(S)]
    for form, b in ((capi.SEQUENTIAL, 0), (capi.CONCURRENT_M, 0), (capi.CONCURRENT_S, 7), (capi.CONCURRENT_S, 0)):
        req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=3)
        C = np.zeros((S, Nt + 1, 2))
        capi.tbpm_correlation(ctx, lat, req, C)
        C = C[..., 0] + 1j * C[..., 1]
        for s in range(S):
            err = np.max(np.abs(C[s] - refs[s])) / abs(refs[s][0])
            assert err <= TOL[prec], (form, b, s, err)
    capi.tbpm_lattice_destroy(lat)


def test_jackson_dos_matches_oracle(capi, ctx):
    lat, ol = make(capi, ctx, kind=1, L=(20, 20), W=0.5, cutoff=7.1)
    S, M, nE = 2, 512, 257
    E = np.linspace(ol.H0 - 0.99 * ol.half_width, ol.H0 + 0.99 * ol.half_width, nE)  # |E~| = 1 is singular
    req = capi.request(n_states=S, precision=0, n_moments=M, dos_method=capi.DOS_JACKSON)
    D = np.zeros((S, nE))
    capi.tbpm_dos(ctx, lat, req, E, D)
    psi = oprop.random_phase_states(ol, 1, S)
    for s in range(S):
        ref = ospec.dos_jackson(oprop.moments(ol, psi[s], psi[s], M), E, ol.H0, ol.half_width)
        assert np.max(np.abs(D[s] - ref)) / np.max(ref) <= TOL[0]
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("form,b", [(2, 5), (3, 0)])
def test_quasi_eigenstates_match_oracle(capi, ctx, form, b):
    lat, ol = make(capi, ctx, kind=1, L=(10, 9), W=1.0, cutoff=4.1)
    E = np.array([-6.0, -1.1, 0.3, 4.2])
    Nt, S = 17, 2
    out = np.zeros((E.size, S, ol.n), np.complex128)
    capi.tbpm_quasi_eigenstates(ctx, lat, capi.request(n_states=S, precision=1, form=form, n_steps=Nt,
                                                       time_block=b, state_seed=8), E, out)
    psi = oprop.random_phase_states(ol, 8, S)
    for s in range(S):
        ref = oqe.qe_concurrent_e(ol, psi[s], E, Nt)
        for k in range(E.size):
            assert np.max(np.abs(out[k, s] - ref[k])) / np.max(np.abs(ref[k])) <= TOL[1]
    capi.tbpm_lattice_destroy(lat)


def test_fermi_operator_matches_exact(capi, ctx):
    lat, ol = make(capi, ctx, kind=1, L=(8, 7), W=1.0, cutoff=3.1)
    S = 2
    mu, kT = ol.H0 + 0.1 * ol.half_width, 0.08 * ol.half_width
    out = np.zeros((S, ol.n), np.complex128)
    capi.tbpm_fermi_apply(ctx, lat, capi.request(n_states=S, precision=1, state_seed=5), mu, kT, False, out)
    psi = oprop.random_phase_states(ol, 5, S)
    for s in range(S):
        ref = R.fermi_operator_exact(ol, psi[s], mu, kT)
        assert np.max(np.abs(out[s] - ref)) / np.max(np.abs(ref)) <= 1e-10
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("prec", [1, 0])
def test_polarization_and_charge_density_match_oracle(capi, ctx, prec):
    lat, ol = make(capi, ctx, kind=1, L=(9, 8), W=1.0, cutoff=3.1)
    S, Nt = 2, 15
    mu = ol.H0 + 0.15 * (ol.E_max - ol.E_min) / 2
    kT = 0.1 * (ol.E_max - ol.E_min) / 2
    q = [0.3, -0.2, 0.0]
    om = np.linspace(0.0, ol.E_max - ol.E_min, 9)
    C = np.zeros((S, Nt + 1), np.complex128)
    Pi = np.zeros((S, om.size), np.complex128)
    capi.tbpm_polarization(ctx, lat, capi.request(n_states=S, precision=prec, form=2, n_steps=Nt, time_block=4,
                                                  state_seed=7), q, mu, kT, om, C, Pi)
    psi = oprop.random_phase_states(ol, 7, S)
    for s in range(S):
        Cref = R.dp_correlation_sequential(ol, psi[s], q, mu, kT, Nt)
        assert np.max(np.abs(C[s] - Cref)) / np.max(np.abs(Cref)) <= TOL_RESP[prec]
    rho = np.zeros((S, ol.n))
    capi.tbpm_charge_density(ctx, lat, capi.request(n_states=S, precision=prec, form=2, n_steps=Nt, time_block=4,
                                                    state_seed=11), mu, kT, rho)
    psi = oprop.random_phase_states(ol, 11, S)
    tau = ocd.cd_default_tau(ol, mu, kT)
    for s in range(S):
        ref = ocd.charge_density_sequential(ol, psi[s], mu, kT, Nt, tau)
        assert np.max(np.abs(rho[s] - ref)) / np.max(np.abs(ref)) <= TOL_RESP[prec]
    capi.tbpm_lattice_destroy(lat)


def test_recreated_lattice_does_not_replay_a_destroyed_lattices_graph(capi, ctx):
    """Moment passes are captured in CUDA graphs from their second call on.  A lattice destroyed
    and created again (often at the same host address, with the same sizes and coefficients)
    must run on its own tap table, not replay the old lattice's graph."""
    desc = capi.lattice_desc(1, (70, 36), t=-2.7, cutoff=7.1, decay=DECAY)
    runs = []
    for _ in range(3):
        lat = capi.tbpm_lattice_create(ctx, desc)
        runs.append([gpu_moments(capi, ctx, lat, 2, 200, 0) for _ in range(3)])
        capi.tbpm_lattice_destroy(lat)
    for r in runs:
        for m in r:
            assert np.array_equal(m, runs[0][0])


EC_CASES = [
    ("honey9x8_c3.1_x_c128", dict(kind=1, L=(9, 8), W=1.0, cutoff=3.1), 0, 1, 2),
    ("honey9x8_c3.1_y_c64", dict(kind=1, L=(9, 8), W=1.0, cutoff=3.1), 1, 0, 2),
    ("honey9x8_c3.1_y_c128", dict(kind=1, L=(9, 8), W=1.0, cutoff=3.1), 1, 1, 2),
    ("square11x9_c2.9_open_x_c128", dict(kind=0, L=(11, 9), t=1.0, W=1.0, pbc=(0, 1, 1), cutoff=2.9, decay=0.6),
     0, 1, 1),
    ("honey10x8_c2.1_vac_y_c128", dict(kind=1, L=(10, 8), W=1.5, vac=0.04, cutoff=2.1), 1, 1, 1),
]


@pytest.mark.parametrize("form,b", [(0, 0), (2, 4), (1, 0)])
@pytest.mark.parametrize("name,spec,direction,prec,S", EC_CASES, ids=[c[0] for c in EC_CASES])
def test_conductivity_matches_oracle(capi, ctx, name, spec, direction, prec, S, form, b):
    """EC in the three forms on long-range lattices: every tap carries its own bond vector in the
    current operator (oracle: brute force over site pairs and images).

    C(t, E) = <J psi(t)|J Psi(E)> / |<psi|Psi(E)>| is a ratio (Eq. dc_corr), so its two factors
    are pinned separately at the plain tolerance, each relative to its own Cauchy-Schwarz bound:
    the overlap <psi|Psi(E)> against |psi| |Psi(E)|, and the numerator (C times the overlap the
    device used) against |J psi| |J Psi(E)|.  C itself and sigma then obey the bound that follows
    from the quotient rule (the reading of the EC tolerance stated in the design notes)."""
    from oracle import conductivity as oec
    lat, ol = make(capi, ctx, **spec)
    E = ol.H0 + np.array([-0.6, 0.05, 0.4]) * (ol.E_max - ol.E_min) / 2
    Nt = 15
    C = np.zeros((S, E.size, Nt + 1), np.complex128)
    sigma = np.zeros((S, E.size))
    ovl = np.zeros((S, E.size), np.complex128)
    capi.tbpm_conductivity_overlap(ctx, lat, capi.request(n_states=S, precision=prec, form=form, n_steps=Nt,
                                                          time_block=b, state_seed=12), direction, E, C, sigma, ovl)
    psi = oprop.random_phase_states(ol, 12, S)
    tol = {0: 3e-5, 1: 1e-10}[prec]
    J = oec.current_operator(ol, direction)
    for s in range(S):
        Cref, qe = oec.ec_correlation_sequential(ol, psi[s], E, Nt, direction)
        sref = oec.conductivity(ol, psi[s], E, Cref, qe)
        ov_ref = qe.conj() @ psi[s]
        ov = np.abs(ov_ref)
        Dn = np.abs(ov_ref.real) / oec.area_per_site(ol.kind)
        for k in range(E.size):
            # the two factors at the plain tolerance
            cs_ov = np.linalg.norm(psi[s]) * np.linalg.norm(qe[k])
            assert abs(np.conj(ovl[s, k]) - ov_ref[k]) <= tol * cs_ov, ("overlap", s, k)
            cs_num = np.linalg.norm(J @ psi[s]) * np.linalg.norm(J @ qe[k])
            num = C[s, k] * abs(ovl[s, k])
            num_ref = Cref[k] * ov[k]
            assert np.max(np.abs(num - num_ref)) <= tol * cs_num, ("numerator", s, k)
            # the quotient: |dC| <= |d num| / |ov| + |C| |d ov| / |ov|
            scale = cs_num / ov[k]
            cond = cs_ov / ov[k]
            err_bound = tol * (scale + np.max(np.abs(Cref[k])) * cond)
            assert np.max(np.abs(C[s, k] - Cref[k])) <= err_bound, ("C", s, k)
            bound = Dn[k] * (np.pi / ol.half_width) * (Nt + 1) * err_bound
            assert abs(sigma[s, k] - sref[k]) <= bound, ("sigma", s, k)
    capi.tbpm_lattice_destroy(lat)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("alpha,beta", [(0, 0), (0, 1)])
def test_optical_conductivity_matches_oracle(capi, ctx, alpha, beta, prec):
    lat, ol = make(capi, ctx, kind=1, L=(9, 8), W=1.0, cutoff=3.1)
    S, Nt, nw = 2, 17, 25
    mu = ol.H0 - 0.1 * (ol.E_max - ol.E_min) / 2
    kT = 0.08 * (ol.E_max - ol.E_min) / 2
    wmax = 1.2 * (ol.E_max - ol.E_min)
    C = np.zeros((S, Nt + 1), np.complex128)
    sig = np.zeros((S, nw), np.complex128)
    capi.tbpm_optical_conductivity(ctx, lat, capi.request(n_states=S, precision=prec, form=2, n_steps=Nt,
                                                          time_block=5, state_seed=6), alpha, beta, mu, kT, wmax, nw,
                                   C, sig)
    psi = oprop.random_phase_states(ol, 6, S)
    for s in range(S):
        Cref = R.oc_correlation_sequential(ol, psi[s], alpha, beta, mu, kT, Nt)
        assert np.max(np.abs(C[s] - Cref)) / np.max(np.abs(Cref)) <= TOL_RESP[prec]
    capi.tbpm_lattice_destroy(lat)


def test_unsupported_calls_and_invalid_descriptions(capi, ctx):
    for kw in (dict(cutoff=2.0, decay=0.0), dict(cutoff=-1.0, decay=1.0), dict(cutoff=13.0, decay=1.0),
               dict(cutoff=0.5, decay=1.0), dict(cutoff=2.0, decay=1.0, path=1)):
        with pytest.raises(capi.TbpmError):
            capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (8, 8), t=-2.7, **kw))
    srv = capi.tbpm_server_create(ctx)
    try:
        with pytest.raises(capi.TbpmError):
            capi.tbpm_submit(srv, capi.lattice_desc(1, (8, 8), t=-2.7, cutoff=2.1, decay=0.5),
                             capi.request(n_states=1, n_moments=64), np.array([0.0]))
    finally:
        capi.tbpm_server_destroy(srv)


def test_fp32_fma_peak_is_a_plausible_device_rate(capi, ctx):
    """The measured FP32 FMA rate that the tap kernel's roofline divides by: positive for both
    forms and below what the device's SMs could issue at 128 FP32 lanes and 3 GHz."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    scalar, packed = capi.tbpm_fp32_fma_peak(ctx)
    bound = sms * 128 * 2 * 3.0e9 / 1e12
    assert 0.0 < scalar < bound and 0.0 < packed < 2 * bound, (scalar, packed, bound)
