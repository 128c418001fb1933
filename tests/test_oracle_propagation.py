"""Pins of the oracle's propagation, moments and spectra.

Pinned against exact diagonalisation (numpy eigh) on lattices of a few hundred
sites, closed-form clean-lattice moments, the invariants the paper relies on
(mu_0 = 1, norm conservation, C(-t) = C(t)*), the paper's operation counts (Tab. I)
and the Nyquist-step identity of the Fourier DOS.
"""
import math

import numpy as np
import pytest

from oracle import lattice, propagate as pr, spectra, cost, bessel
from oracle.lattice import SQUARE, HONEYCOMB, CUBIC


def ed(lat, psi):
    E, U = np.linalg.eigh(lat.H.toarray())
    w = np.abs(U.conj().T @ psi) ** 2
    return E, w


def ed_moments(lat, w, E, M):
    x = (E - lat.H0) / lat.half_width
    return np.array([np.sum(w * np.cos(n * np.arccos(x))) for n in range(M)])


@pytest.fixture(scope="module")
def square16():
    """16x16 square lattice, t=1, V in [-0.5, 0.5]: the exact-diagonalisation check size."""
    lat = lattice.build_lattice(SQUARE, (16, 16, 1), t=1.0, W=1.0, seed=0x7B1A5)
    psi = pr.random_phase_states(lat, 1, 1)[0]
    E, w = ed(lat, psi)
    return lat, psi, E, w


@pytest.fixture(scope="module")
def honey10():
    lat = lattice.build_lattice(HONEYCOMB, (10, 10, 1), t=-2.7, W=1.0, seed=0x7B1A5)
    psi = pr.random_phase_states(lat, 7, 1)[0]
    E, w = ed(lat, psi)
    return lat, psi, E, w


def test_random_phase_state_normalised(square16):
    lat, psi, _, _ = square16
    assert abs(np.vdot(psi, psi) - 1.0) < 1e-15
    assert np.allclose(np.abs(psi), 1.0 / 16.0, rtol=1e-15, atol=0)


@pytest.mark.parametrize("fx", ["square16", "honey10"])
def test_moments_equal_exact_diagonalisation(fx, request):
    lat, psi, E, w = request.getfixturevalue(fx)
    M = 512
    mu = pr.moments(lat, psi, psi, M)
    assert np.max(np.abs(mu - ed_moments(lat, w, E, M))) < 1e-12
    assert abs(mu[0] - 1.0) < 1e-15


@pytest.mark.parametrize("fx", ["square16", "honey10"])
def test_doubling_equals_plain_moments(fx, request):
    """The cost-halving identity (Eq. cheby_prod) with the factor 2 restored."""
    lat, psi, _, _ = request.getfixturevalue(fx)
    M = 400
    a = pr.moments(lat, psi, psi, M)
    b = pr.moments_doubling(lat, psi, M)
    assert np.max(np.abs(a - b)) < 1e-13


def test_doubling_printed_form_is_wrong_without_factor_two(square16):
    """Eq. cheby-moment as printed (no factor 2) disagrees with the plain moments."""
    lat, psi, _, _ = square16
    phis = list(pr.chebyshev_states(lat, psi, 6))
    m = pr.moments(lat, psi, psi, 10)
    printed = np.vdot(phis[3], phis[3]) - m[0]
    restored = 2 * np.vdot(phis[3], phis[3]) - m[0]
    assert abs(restored - m[6]) < 1e-14
    assert abs(printed - m[6]) > 1e-3


@pytest.mark.parametrize("fx", ["square16", "honey10"])
def test_sequential_correlation_equals_exact(fx, request):
    lat, psi, E, w = request.getfixturevalue(fx)
    Nt = 60
    C, norms = pr.correlation_sequential(lat, psi, Nt, return_norms=True)
    tau = math.pi / lat.half_width
    Ced = np.array([np.sum(w * np.exp(-1j * E * j * tau)) for j in range(Nt + 1)])
    assert np.max(np.abs(C - Ced)) < 1e-12
    assert np.max(np.abs(norms - 1.0)) < 1e-12


def test_concurrent_forms_equal_sequential(square16):
    """Sec. III accuracy claim (eps_inf 8.3e-14 for C): moment-based and state-based forms
    reproduce the sequential correlation."""
    lat, psi, _, _ = square16
    Nt = 100
    Cs = pr.correlation_sequential(lat, psi, Nt)
    M = bessel.truncation_order(Nt * math.pi)
    mu = pr.moments(lat, psi, psi, M)
    Cm = pr.correlation_from_moments(mu, Nt, math.pi, lat.H0 / lat.half_width)
    assert np.max(np.abs(Cm - Cs)) < 1e-12
    for b in (1, 4, 13, 100):
        Cb, states = pr.propagate_state_blocks(lat, psi, Nt, b)
        assert np.max(np.abs(Cb - Cs)) < 1e-12
        assert np.max(np.abs(np.linalg.norm(states, axis=1) - 1.0)) < 1e-12


def test_hermitian_symmetry_of_correlation(honey10):
    """C(-t) = C(t)* (Sec. III), checked by actually propagating backwards."""
    lat, psi, _, _ = honey10
    Cf = pr.correlation_sequential(lat, psi, 40)
    Cb = pr.correlation_backward(lat, psi, 40)
    assert np.max(np.abs(Cb - np.conj(Cf))) < 1e-13


def test_phase_factor_matters_with_offset():
    """With a shifted spectrum (H0 != 0) the exp(-i H0 t) factor is needed to match ED."""
    import scipy.sparse as sp
    lat = lattice.build_lattice(SQUARE, (6, 6, 1), t=1.0, W=0.0, seed=1)
    # add a uniform on-site offset 0.8 and move the bounds with it
    H = lat.H + sp.identity(lat.n) * 0.8
    lat.H = H.tocsr()
    lat.E_max += 0.8
    lat.E_min += 0.8
    lat.H0 = (lat.E_max + lat.E_min) / 2
    psi = pr.random_phase_states(lat, 3, 1)[0]
    E, w = ed(lat, psi)
    tau = math.pi / lat.half_width
    C = pr.correlation_sequential(lat, psi, 20)
    Ced = np.array([np.sum(w * np.exp(-1j * E * j * tau)) for j in range(21)])
    assert np.max(np.abs(C - Ced)) < 1e-12


@pytest.mark.parametrize("kind,L,z", [(SQUARE, (12, 10, 1), 4), (HONEYCOMB, (6, 8, 1), 3),
                                      (CUBIC, (4, 6, 4), 6)])
def test_clean_ldos_closed_forms(kind, L, z):
    """Clean periodic lattices: the LDOS moments of any site equal the band average
    (1/N) sum_k T_n(E(k)/|H|) with the analytic bands; mu_2 = 2 z t^2/|H|^2 - 1; odd moments
    vanish on bipartite lattices with even sides."""
    t = -1.7
    lat = lattice.build_lattice(kind, L, t=t)
    s = lat.half_width
    r = [0, lat.n // 2 + 1]
    states = pr.site_states(lat, r)
    M = 48
    Lx, Ly, Lz = L
    if kind == SQUARE:
        kx, ky = np.meshgrid(2 * np.pi * np.arange(Lx) / Lx, 2 * np.pi * np.arange(Ly) / Ly)
        bands = [2 * t * (np.cos(kx) + np.cos(ky))]
    elif kind == CUBIC:
        kx, ky, kz = np.meshgrid(2 * np.pi * np.arange(Lx) / Lx, 2 * np.pi * np.arange(Ly) / Ly,
                                 2 * np.pi * np.arange(Lz) / Lz)
        bands = [2 * t * (np.cos(kx) + np.cos(ky) + np.cos(kz))]
    else:
        k1, k2 = np.meshgrid(2 * np.pi * np.arange(Lx) / Lx, 2 * np.pi * np.arange(Ly) / Ly)
        f = np.abs(1 + np.exp(1j * k1) + np.exp(1j * k2))
        bands = [abs(t) * f, -abs(t) * f]
    Ek = np.concatenate([b.ravel() for b in bands])
    x = Ek / s
    ref = np.array([np.mean(np.cos(n * np.arccos(np.clip(x, -1, 1)))) for n in range(M)])
    for st in states:
        mu = pr.moments(lat, st, st, M)
        assert np.max(np.abs(mu - ref)) < 1e-13
        assert abs(mu[2] - (2 * z * t * t / s ** 2 - 1)) < 1e-14
        assert np.max(np.abs(mu[1::2])) < 1e-14


def test_vacancy_lattice_matches_exact_diagonalisation():
    lat = lattice.build_lattice(HONEYCOMB, (9, 8, 1), t=-2.7, W=2.0, vacancy_frac=0.05, seed=21)
    psi = pr.random_phase_states(lat, 4, 1)[0]
    E, w = ed(lat, psi)
    mu = pr.moments(lat, psi, psi, 200)
    assert np.max(np.abs(mu - ed_moments(lat, w, E, 200))) < 1e-12


# ---------------------------------------------------------------- spectra

def test_jackson_factors_closed_forms():
    """g_0 = 1 and g_1 = cos(pi/(M+1)) for the Jackson kernel (Weisse et al. 2006, Sec. II.C)."""
    for M in (2, 7, 64, 1000):
        g = spectra.jackson_factors(M)
        assert abs(g[0] - 1.0) < 1e-15
        assert abs(g[1] - math.cos(math.pi / (M + 1))) < 1e-14
        assert np.all(g > -1e-15) and np.all(np.diff(g) <= 1e-15)


def test_jackson_dos_integral_and_positivity(square16):
    """Chebyshev-Gauss quadrature at N_E >= M nodes integrates the Jackson DOS exactly:
    int D dE = g_0 mu_0 = 1.  The Jackson-damped series of a positive measure is >= 0."""
    lat, psi, E, w = square16
    M = 256
    mu = pr.moments(lat, psi, psi, M)
    NE = 512
    xk = np.cos(np.pi * (np.arange(NE) + 0.5) / NE)
    energies = lat.H0 + lat.half_width * xk
    D = spectra.dos_jackson(mu, energies, lat.H0, lat.half_width)
    weight = np.pi * lat.half_width * np.sqrt(1 - xk ** 2) / NE
    assert abs(np.sum(D * weight) - 1.0) < 1e-12
    assert D.min() > -1e-12


def test_jackson_dos_of_exact_moments_peaks_at_eigenvalues():
    """Two-level check: for mu_n = T_n(x0) (a single eigenvalue) the damped series peaks at x0."""
    M, x0 = 400, 0.37
    mu = np.cos(np.arange(M) * np.arccos(x0)).astype(complex)
    grid = np.linspace(-0.99, 0.99, 4001)
    D = spectra.dos_jackson(mu, grid, 0.0, 1.0)
    assert abs(grid[np.argmax(D)] - x0) < 2e-3


def test_fourier_dos_nyquist_identity(square16):
    """With C(t_j) from ED, the sampled-and-windowed transform equals the ED spectrum convolved
    with the window's kernel K(e) = (tau/2pi)[w_0 + 2 sum_j w_j cos(e t_j)]; one period of the
    DOS (2|H| at tau~ = pi, the Nyquist step) integrates to w_0 C(0) = 1."""
    lat, psi, E, w = square16
    Nt = 64
    C = pr.correlation_sequential(lat, psi, Nt)
    tau = math.pi / lat.half_width
    grid = lat.H0 + lat.half_width * np.linspace(-1, 1, 301)[:-1]
    for kind in (spectra.WINDOW_NONE, spectra.WINDOW_HANN):
        D = spectra.dos_fourier(C, tau, grid, kind)
        wj = spectra.window(Nt, kind)
        j = np.arange(1, Nt + 1)
        K = lambda e: tau / (2 * np.pi) * (wj[0] + 2 * np.sum(wj[1:] * np.cos(e * j * tau)))
        ref = np.array([np.sum(w * np.array([K(g - Ek) for Ek in E])) for g in grid[::15]])
        assert np.max(np.abs(D[::15] - ref)) < 1e-11
        period = 2 * lat.half_width
        assert abs(np.sum(D) * period / grid.size - wj[0]) < 1e-11


# ---------------------------------------------------------------- Tab. I operation counts

def test_operation_counts_match_table_one(square16):
    lat, psi, _, _ = square16
    Nt = 30
    ops = pr.OpCounter()
    pr.correlation_sequential(lat, psi, Nt, ops=ops)
    want = cost.dos_sequential_counts(Nt)
    assert (ops.amxsy, ops.axpy, ops.dot) == (want["amxsy"], want["axpy"], want["dot"])
    assert want["amxsy"] == Nt * 20

    M = bessel.truncation_order(Nt * math.pi)
    M += M % 2
    ops = pr.OpCounter()
    pr.moments_doubling(lat, psi, M, ops=ops)
    # Tab. I: N(t_tot)/2 matrix-vector products (plus the free T_0 term) and N(t_tot) dots
    assert ops.amxsy - 1 == M // 2
    assert ops.dot == M

    for b in (1, 5, 30):
        ops = pr.OpCounter()
        pr.propagate_state_blocks(lat, psi, Nt, b, ops=ops)
        want = cost.block_counts(Nt, b)
        assert (ops.amxsy, ops.axpy, ops.dot) == (want["amxsy"], want["axpy"], want["dot"])
    # b = 1 is the sequential form
    assert cost.block_counts(Nt, 1) == {k: v for k, v in cost.dos_sequential_counts(Nt).items()
                                         if k != "states"}


def test_block_size_model_has_interior_optimum():
    """Sec. II.B: C(b) first falls then rises once the b-way axpy outweighs the saved amxsy."""
    Nt = 1024
    b = cost.b_opt(Nt, t_amxsy=1.0, t_axpy=0.2, b_max=256)
    assert 4 < b < 256
    cb = [cost.block_cost(Nt, x, 1.0, 0.2) for x in (1, b, 256)]
    assert cb[1] < cb[0] and cb[1] < cb[2]
    assert abs(cost.amdahl(0.77, 1e9) - 1 / 0.23) < 1e-6
    assert cost.amdahl(1.0, 3.0) == pytest.approx(3.0)
