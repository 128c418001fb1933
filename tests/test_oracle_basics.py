"""Pins of the oracle's building blocks: Philox, lattices, Bessel coefficients, truncation.

Each test checks the oracle against something other than itself: published
known-answer vectors, hand-derived neighbour tables, mpmath/scipy Bessel values,
closed-form identities, and the expansion-load figures the paper prints (Sec. II.A).
"""
import math
import os

import numpy as np
import pytest

from conftest import GOLDEN
from oracle import philox, lattice, bessel
from oracle.lattice import SQUARE, HONEYCOMB, CUBIC

KINDS = {"square": SQUARE, "honeycomb": HONEYCOMB, "cubic": CUBIC}


def read_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(v, 16) for v in line.split()]
            rows.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return rows


def read_neighbours():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "neighbours.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            if line.startswith("lattice"):
                p = line.split()
                cur = (KINDS[p[1]], tuple(int(v) for v in p[2:5]), tuple(int(v) for v in p[5:8]), {})
                cases.append(cur)
            else:
                site, rest = line.split(":")
                cur[3][int(site)] = [int(v) for v in rest.split()]
    return cases


def test_philox_known_answers():
    rows = read_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = philox.philox4x32_10(ctr, key)
        assert tuple(int(v) for v in got) == want


def test_philox_vectorised_equals_scalar():
    idx = np.arange(50, dtype=np.uint64) * np.uint64(2654435761)
    vec = philox.draw_u32(0x123456789ABCDEF, idx, 2, 5)
    for k in range(50):
        one = philox.draw_u32(0x123456789ABCDEF, np.array([idx[k]]), 2, 5)
        assert vec[k] == one[0]


@pytest.mark.parametrize("case", range(4))
def test_neighbour_tables_golden(case):
    kind, L, pbc, table = read_neighbours()[case]
    nbr = lattice.neighbour_table(kind, L, pbc)
    for site, want in table.items():
        assert nbr[site].tolist() == want, (kind, L, pbc, site)


@pytest.mark.parametrize("kind,L", [(SQUARE, (5, 4, 1)), (HONEYCOMB, (4, 3, 1)), (CUBIC, (3, 4, 5))])
def test_hamiltonian_symmetric_and_bipartite_counts(kind, L):
    lat = lattice.build_lattice(kind, L, t=-1.3, W=0.7, seed=11)
    H = lat.H.toarray()
    assert np.array_equal(H, H.T)
    z = lattice.COORDINATION[kind]
    assert np.all(lat.degree == z)
    off = H - np.diag(np.diag(H))
    assert np.allclose(np.abs(off).sum(axis=1), z * 1.3)


def test_open_boundary_degrees():
    lat = lattice.build_lattice(SQUARE, (4, 3, 1), t=1.0, pbc=(0, 0, 1))
    deg = lat.degree.reshape(3, 4)
    assert deg[0, 0] == 2 and deg[1, 1] == 4 and deg[0, 1] == 3


def test_disorder_distribution():
    V = lattice.disorder_potential(0x7B1A5, 2.0, 200000)
    assert V.min() >= -1.0 and V.max() < 1.0
    assert abs(V.mean()) < 0.01
    assert abs(V.var() - 4.0 / 12.0) < 0.01
    # every value is W times a multiple of 2^-24 (24-bit uniform grid)
    q = (V / 2.0 + 0.5) * 2.0 ** 24
    assert np.all(q == np.round(q))


def test_vacancies_fraction_and_compaction():
    lat = lattice.build_lattice(HONEYCOMB, (64, 64, 1), t=-2.7, vacancy_frac=0.05, seed=3)
    frac = 1.0 - lat.n / lat.n_full
    assert abs(frac - 0.05) < 0.01
    assert np.array_equal(np.flatnonzero(lat.compact >= 0), np.flatnonzero(lat.active))
    assert np.array_equal(lat.compact[lat.active], np.arange(lat.n))
    # no bond touches a vacant site; degrees never exceed z
    assert lat.H.shape == (lat.n, lat.n)
    assert np.all(lat.degree <= 3)
    assert lattice.vacancy_threshold(0.01) == 42949672


@pytest.mark.parametrize("kind,L,W", [(SQUARE, (12, 10, 1), 1.5), (HONEYCOMB, (8, 7, 1), 0.9),
                                      (CUBIC, (5, 4, 3), 2.0)])
def test_gershgorin_bounds_contain_spectrum(kind, L, W):
    lat = lattice.build_lattice(kind, L, t=1.0, W=W, seed=9)
    E = np.linalg.eigvalsh(lat.H.toarray())
    assert lat.E_min <= E.min() and E.max() <= lat.E_max
    x = (E - lat.H0) / lat.half_width
    assert np.all(np.abs(x) < 1.0 / 1.005)


def test_clean_bounds_closed_form():
    lat = lattice.build_lattice(HONEYCOMB, (6, 6, 1), t=-2.7)
    assert lat.E_max == pytest.approx(8.1, rel=1e-15) and lat.E_min == -lat.E_max
    assert lat.H0 == 0.0
    assert lat.half_width == pytest.approx(1.01 * 8.1, rel=1e-15)


# ---------------------------------------------------------------- Bessel coefficients

@pytest.mark.parametrize("x", [0.3, math.pi, 17.0, 4 * math.pi, 250.0, 1254 * math.pi])
def test_bessel_matches_scipy(x):
    from scipy.special import jv
    n = int(x) + 60
    J = bessel.bessel_j_sequence(x, n)
    ref = jv(np.arange(n + 1), x)
    assert np.max(np.abs(J - ref)) < 2e-14 + 1e-16 * x


def test_bessel_matches_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for x, ns in ((math.pi, (0, 1, 5, 19, 25)), (100.0, (0, 7, 99, 140)),
                  (1254 * math.pi, (0, 1, 100, 2000, 3934, 4039))):
        J = bessel.bessel_j_sequence(x, max(ns) + 1)
        for n in ns:
            ex = float(mpmath.besselj(n, mpmath.mpf(x)))
            assert abs(J[n] - ex) < 5e-16 + 1e-15 * abs(ex), (x, n)


def test_bessel_negative_argument_and_zero():
    J = bessel.bessel_j_sequence(-3.0, 10)
    Jp = bessel.bessel_j_sequence(3.0, 10)
    assert np.allclose(J, Jp * (-1.0) ** np.arange(11), atol=0, rtol=0)
    assert bessel.bessel_j_sequence(0.0, 4).tolist() == [1.0, 0.0, 0.0, 0.0, 0.0]


@pytest.mark.parametrize("tau", [0.7, math.pi, 10.0, 40 * math.pi])
def test_jacobi_anger_at_band_edges(tau):
    """sum_n c_n(tau) T_n(x) = exp(-i x tau) at x = +-1, where T_n(1) = 1, T_n(-1) = (-1)^n."""
    N = bessel.truncation_order(tau)
    c = bessel.cheb_coefficients(tau, N)
    n = np.arange(N)
    assert abs(np.sum(c) - np.exp(-1j * tau)) < 1e-13
    assert abs(np.sum(c * (-1.0) ** n) - np.exp(1j * tau)) < 1e-13
    # and at an interior point, against the trigonometric T_n
    x = 0.3141
    assert abs(np.sum(c * np.cos(n * np.arccos(x))) - np.exp(-1j * x * tau)) < 1e-13


def test_truncation_matches_paper_expansion_load():
    """Sec. II.A / Fig. 2(b): R(pi) is about 6 and falls to about 1/2, 1/3, 1/4, 1/5 of that
    value at tau~ = 4pi, 10pi, 25pi, 100pi."""
    assert bessel.truncation_order(math.pi) == 20
    R0 = bessel.expansion_load(math.pi)
    assert abs(R0 - 6.0) < 0.5
    for k, frac in ((4, 1 / 2), (10, 1 / 3), (25, 1 / 4), (100, 1 / 5)):
        r = bessel.expansion_load(k * math.pi) / R0
        assert abs(r - frac) < 0.03, (k, r)
    # R tends to 1 at long times (Sec. II.A): theoretical DOS-M speedup ~ R(pi)/R(inf) ~ 6
    assert 1.0 < bessel.expansion_load(2000 * math.pi) < 1.1


def test_truncation_definition_edges():
    tau = 4 * math.pi
    N = bessel.truncation_order(tau)
    c = np.abs(bessel.cheb_coefficients(tau, N + 40))
    assert c[N - 1] > bessel.ETA and np.all(c[N:] <= bessel.ETA)


def test_theoretical_dos_speedup_about_12():
    """Sec. III: moment-based DOS with the cost halving is ~12x cheaper than sequential
    (N_t N(pi) SpMVs versus N(N_t pi)/2) at N_t = 4096."""
    Nt = 4096
    ratio = Nt * bessel.truncation_order(math.pi) / (bessel.truncation_order(Nt * math.pi) / 2)
    assert 11.0 < ratio < 13.5
