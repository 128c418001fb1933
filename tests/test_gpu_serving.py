"""Serving: continuous batching of DOS/LDOS requests (tbpm_submit / tbpm_wait).

Checks that every served result matches the oracle, that a batched result equals the direct API's
result within the path tolerance and a direct-lane result equals it bit for bit, that a
request's result is bit-identical alone and inside a mix of other requests, that admission
follows the HBM budget, that requests submitted while others run join the batch and finish
first when they are short, and that waits time out and servers cancel cleanly.
"""
import time

import numpy as np
import pytest

from oracle import lattice as olat, propagate as oprop, spectra as ospec

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


def energies(n=200, half=9.0):
    return np.linspace(-half, half, n)


CASES = [
    ("square_c64_S3", dict(kind=0, L=(48, 40), t=1.0, W=1.0, seed=3), dict(n_states=3, precision=0, n_moments=256)),
    ("honey_c64_S8", dict(kind=1, L=(64, 30), t=-2.7, W=0.5, seed=4), dict(n_states=8, precision=0, n_moments=400)),
    ("cubic_c128_S2", dict(kind=2, L=(9, 8, 7), t=1.0, W=2.0, seed=5), dict(n_states=2, precision=1, n_moments=200)),
    ("honey_vac_c64", dict(kind=1, L=(40, 40), t=-2.7, W=1.0, vacancy_frac=0.02, seed=6),
     dict(n_states=4, precision=0, n_moments=300)),
    ("square_ldos_c64", dict(kind=0, L=(300, 3), t=1.0, W=1.0, seed=7),
     dict(sites=[0, 17, 599, 899], precision=0, n_moments=128)),
    ("honey_long_lines", dict(kind=1, L=(1500, 4), t=-2.7, W=1.0, seed=8), dict(n_states=16, precision=0, n_moments=64)),
]


# requests of at least 2^21 site-states run in a direct lane (own stream, the direct path's kernels)
LANE_CASES = [
    ("square_lane_S1", dict(kind=0, L=(1500, 1500), t=1.0, W=1.0, seed=21), dict(n_states=1, precision=0, n_moments=64)),
    ("honey_lane_ldos", dict(kind=1, L=(768, 768), t=-2.7, W=0.5, seed=22),
     dict(sites=[5, 100000, 1179647], precision=0, n_moments=96)),
    ("honey_lane_S8_fused", dict(kind=1, L=(400, 330), t=-2.7, W=0.0, seed=23), dict(n_states=8, precision=0, n_moments=160)),
]


def direct_dos(capi, ctx, ldesc, rkw, E):
    lat = capi.tbpm_lattice_create(ctx, ldesc)
    req = capi.request(dos_method=capi.DOS_JACKSON, **rkw)
    D = np.zeros((req.n_states, E.size))
    capi.tbpm_dos(ctx, lat, req, E, D)
    capi.tbpm_lattice_destroy(lat)
    return D


def test_served_results_match_direct_api(capi, ctx):
    srv = capi.tbpm_server_create(ctx)
    E = energies()
    try:
        tickets = []
        for name, lk, rk in CASES:
            ld = capi.lattice_desc(**lk)
            req = capi.request(**rk)
            tickets.append((name, ld, rk, capi.tbpm_submit(srv, ld, req, E)))
        for name, ld, rk, t in tickets:
            S = len(rk["sites"]) if "sites" in rk else rk["n_states"]
            D = np.zeros((S, E.size))
            capi.tbpm_wait(srv, t, D)
            ref = direct_dos(capi, ctx, ld, rk, E)
            err = np.max(np.abs(D - ref)) / np.max(np.abs(ref))
            assert err <= TOL[rk["precision"]], (name, err)
    finally:
        capi.tbpm_server_destroy(srv)


def oracle_dos(lk, rk, E):
    """The oracle's Jackson DOS of the oracle's moments for one served request."""
    lk = dict(lk)
    kind, L = lk.pop("kind"), tuple(lk.pop("L"))
    ol = olat.build_lattice(kind, L + (1,) * (3 - len(L)), t=lk.get("t", 1.0), W=lk.get("W", 0.0),
                            vacancy_frac=lk.get("vacancy_frac", 0.0), seed=lk.get("seed", 0))
    if "sites" in rk:
        psi = oprop.site_states(ol, rk["sites"])
    else:
        psi = oprop.random_phase_states(ol, rk.get("state_seed", 1), rk["n_states"])
    M = rk["n_moments"]
    return np.stack([ospec.dos_jackson(oprop.moments(ol, p, p, M), E, ol.H0, ol.half_width) for p in psi])


@pytest.mark.parametrize("recon", ["fp64", "tensor"])
def test_served_results_match_oracle(capi, ctx, recon):
    """Every served DOS (square, honeycomb, cubic, vacancies, LDOS, complex64 and complex128, 1 to
    16 states) against the oracle's Jackson DOS of the oracle's moments: max_E |dD| / max_E D <=
    1e-5 for complex64, 1e-11 for complex128 with the FP64 reconstruction (1e-5 through the
    bf16 x3 tensor-core reconstruction)."""
    E = energies()
    srv = capi.tbpm_server_create(ctx, recon=capi.RECON_TENSOR if recon == "tensor" else capi.RECON_FP64)
    try:
        tickets = [(name, lk, rk, capi.tbpm_submit(srv, capi.lattice_desc(**lk), capi.request(**rk), E))
                   for name, lk, rk in CASES + LANE_CASES]
        for name, lk, rk, t in tickets:
            S = len(rk["sites"]) if "sites" in rk else rk["n_states"]
            D = np.zeros((S, E.size))
            capi.tbpm_wait(srv, t, D)
            ref = oracle_dos(lk, rk, E)
            tol = TOL[rk["precision"]] if recon == "fp64" else 1e-5
            for s in range(S):
                err = np.max(np.abs(D[s] - ref[s])) / np.max(np.abs(ref[s]))
                assert err <= tol, (name, s, err)
    finally:
        capi.tbpm_server_destroy(srv)


def test_lane_results_equal_the_direct_api_bit_for_bit(capi, ctx):
    """A direct-lane request runs the same kernels as tbpm_dos on its own stream: its DOS equals
    the direct call's bit for bit, also while batched requests and other lanes run beside it."""
    E = energies()
    srv = capi.tbpm_server_create(ctx)
    try:
        tickets = [(lk, rk, capi.tbpm_submit(srv, capi.lattice_desc(**lk), capi.request(**rk), E))
                   for _, lk, rk in LANE_CASES + CASES[:3]]
        for lk, rk, t in tickets[:len(LANE_CASES)]:
            S = len(rk["sites"]) if "sites" in rk else rk["n_states"]
            D = np.zeros((S, E.size))
            capi.tbpm_wait(srv, t, D)
            assert np.array_equal(D, direct_dos(capi, ctx, capi.lattice_desc(**lk), rk, E))
        for lk, rk, t in tickets[len(LANE_CASES):]:
            S = len(rk["sites"]) if "sites" in rk else rk["n_states"]
            capi.tbpm_wait(srv, t, np.zeros((S, E.size)))
    finally:
        capi.tbpm_server_destroy(srv)


def test_alone_and_in_mix_bit_identical(capi, ctx):
    E = energies(150)
    target_l = capi.lattice_desc(1, (70, 50), t=-2.7, W=1.0, seed=11)
    target_r = dict(n_states=5, precision=0, n_moments=320, state_seed=77)
    srv = capi.tbpm_server_create(ctx)
    try:
        t = capi.tbpm_submit(srv, target_l, capi.request(**target_r), E)
        alone = np.zeros((5, E.size))
        capi.tbpm_wait(srv, t, alone)
        others = []
        for k, (name, lk, rk) in enumerate(CASES):
            others.append(capi.tbpm_submit(srv, capi.lattice_desc(**lk), capi.request(**rk), E))
            if k == 2:
                t = capi.tbpm_submit(srv, target_l, capi.request(**target_r), E)
        mixed = np.zeros((5, E.size))
        capi.tbpm_wait(srv, t, mixed)
        for o, (name, lk, rk) in zip(others, CASES):
            S = len(rk["sites"]) if "sites" in rk else rk["n_states"]
            capi.tbpm_wait(srv, o, np.zeros((S, E.size)))
        assert np.array_equal(alone, mixed)
    finally:
        capi.tbpm_server_destroy(srv)


def test_short_requests_join_and_finish_first(capi, ctx):
    E = energies(64)
    srv = capi.tbpm_server_create(ctx)
    try:
        # a direct-lane request of ~1.4e11 site-updates (a few hundred ms on the fused pass)
        long_t = capi.tbpm_submit(srv, capi.lattice_desc(1, (2048, 1024), t=-2.7, W=0.0),
                                  capi.request(n_states=8, precision=0, n_moments=8192), E)
        time.sleep(0.05)
        shorts = [capi.tbpm_submit(srv, capi.lattice_desc(0, (32, 32), t=1.0, W=1.0, seed=s),
                                   capi.request(n_states=1, precision=0, n_moments=64), E) for s in range(5)]
        lat_short = [capi.tbpm_wait(srv, s, np.zeros((1, E.size)))[2] for s in shorts]
        with pytest.raises(capi.TbpmError):
            capi.tbpm_wait(srv, long_t, np.zeros((8, E.size)), timeout_us=0)
        lat_long = capi.tbpm_wait(srv, long_t, np.zeros((8, E.size)))[2]
        assert max(lat_short) < lat_long
        assert capi.tbpm_server_stats(srv)["completed"] >= 6
    finally:
        capi.tbpm_server_destroy(srv)


def test_admission_by_footprint(capi, ctx):
    E = energies(32)
    srv = capi.tbpm_server_create(ctx, hbm_budget_bytes=32 << 20)
    try:
        big = capi.tbpm_submit(srv, capi.lattice_desc(1, (2048, 1024), t=-2.7),
                               capi.request(n_states=8, precision=0, n_moments=16), E)
        small = [capi.tbpm_submit(srv, capi.lattice_desc(0, (64, 64), t=1.0, W=1.0, seed=s),
                                  capi.request(n_states=2, precision=0, n_moments=32), E) for s in range(4)]
        with pytest.raises(capi.TbpmError) as e:
            capi.tbpm_wait(srv, big, np.zeros((8, E.size)))
        assert e.value.status == -2
        for s in small:
            capi.tbpm_wait(srv, s, np.zeros((2, E.size)))
        st = capi.tbpm_server_stats(srv)
        assert st["reserved_bytes"] == 0 and st["budget_bytes"] == 32 << 20
    finally:
        capi.tbpm_server_destroy(srv)


def test_invalid_submissions_and_cancel(capi, ctx):
    E = energies(16)
    srv = capi.tbpm_server_create(ctx)
    with pytest.raises(capi.TbpmError):
        capi.tbpm_submit(srv, capi.lattice_desc(0, (8, 8)), capi.request(n_states=1, n_moments=7), E)
    with pytest.raises(capi.TbpmError):
        capi.tbpm_wait(srv, 123456, np.zeros((1, 16)))
    for s in range(6):
        capi.tbpm_submit(srv, capi.lattice_desc(1, (512, 512), t=-2.7, seed=s),
                         capi.request(n_states=4, precision=0, n_moments=2048), E)
    capi.tbpm_server_destroy(srv)  # cancels what is queued or running; must not hang
