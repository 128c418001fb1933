"""Pins of the long-range hopping lattices of the oracle (oracle/lattice.py, cutoff > 0): the
stand-in for the paper's dense Hamiltonians of density D_H = 60..230 (Sec. II.B, Sec. IV)."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lattice as olat

DECAY = 0.3187
SQ3 = math.sqrt(3.0)
A1 = np.array([1.5, SQ3 / 2, 0.0])
A2 = np.array([1.5, -SQ3 / 2, 0.0])


def _t(r, t=-2.7, decay=DECAY):
    return t * np.exp(-(r - 1.0) / decay)


@pytest.mark.parametrize("kind,L,pbc,vac", [
    (olat.HONEYCOMB, (5, 4, 1), (1, 1, 1), 0.0), (olat.HONEYCOMB, (6, 3, 1), (0, 1, 1), 0.1),
    (olat.HONEYCOMB, (2, 2, 1), (1, 1, 1), 0.0), (olat.SQUARE, (5, 6, 1), (1, 0, 1), 0.0),
    (olat.SQUARE, (1, 4, 1), (1, 1, 1), 0.0), (olat.CUBIC, (3, 4, 2), (1, 1, 1), 0.05),
    (olat.CUBIC, (4, 3, 3), (0, 1, 0), 0.0)])
def test_cutoff_one_is_the_nearest_neighbour_lattice(kind, L, pbc, vac):
    """0 < r <= 1.2 keeps exactly the nearest neighbours, with t(1) = t: the same H as the
    nearest-neighbour lattice (images that coincide add up on both sides)."""
    nn = olat.build_lattice(kind, L, t=-1.3, W=0.7, vacancy_frac=vac, seed=5, pbc=pbc)
    lr = olat.build_lattice(kind, L, t=-1.3, W=0.7, vacancy_frac=vac, seed=5, pbc=pbc, cutoff=1.2, decay=0.5)
    d = (nn.H - lr.H).tocoo()
    assert lr.n == nn.n and (d.nnz == 0 or np.max(np.abs(d.data)) < 4e-15)  # t(r) with r = 1 to rounding
    assert np.array_equal(np.asarray(lr.degree), np.asarray(nn.degree))
    assert abs(lr.E_max - nn.E_max) < 1e-14 and abs(lr.E_min - nn.E_min) < 1e-14


def test_graphene_neighbour_shells():
    """Textbook multiplicities of the first ten neighbour shells of graphene (distances 1, sqrt3,
    2, sqrt7, 3, sqrt12, sqrt13, 4, sqrt19, sqrt21): 3, 6, 3, 6, 6, 6, 6, 3, 6, 12."""
    r2 = [1, 3, 4, 7, 9, 12, 13, 16, 19, 21]
    mult = [3, 6, 3, 6, 6, 6, 6, 3, 6, 12]
    prev = 0
    for k in range(len(r2)):
        cutoff = math.sqrt(r2[k]) + 0.05
        lat = olat.build_lattice(olat.HONEYCOMB, (14, 14, 1), t=1.0, cutoff=cutoff, decay=1.0)
        deg = np.asarray(lat.degree)
        assert np.all(deg == deg[0])
        assert deg[0] - prev == mult[k], (k, deg[0], prev)
        prev = deg[0]


def _count_infinite(kind, cutoff):
    """Sites of the infinite lattice within the cutoff of site 0 (A for the honeycomb)."""
    R = int(cutoff) + 2
    n = 0
    if kind == olat.HONEYCOMB:
        for m, k, s in itertools.product(range(-R, R + 1), range(-R, R + 1), (0, 1)):
            r = np.linalg.norm(m * A1 + k * A2 + s * np.array([1.0, 0, 0]))
            n += 1e-9 < r <= cutoff
    else:
        rz = range(-R, R + 1) if kind == olat.CUBIC else (0,)
        for m, k, q in itertools.product(range(-R, R + 1), range(-R, R + 1), rz):
            r = math.sqrt(m * m + k * k + q * q)
            n += 1e-9 < r <= cutoff
    return n


@pytest.mark.parametrize("kind,L,cutoff,dh", [(olat.HONEYCOMB, (14, 14, 1), 5.1, 61),
                                              (olat.HONEYCOMB, (18, 18, 1), 7.1, 124),
                                              (olat.HONEYCOMB, (24, 24, 1), 9.7, 235),
                                              (olat.SQUARE, (16, 15, 1), 4.5, None),
                                              (olat.CUBIC, (7, 8, 6), 2.3, None)])
def test_density_matches_the_infinite_lattice(kind, L, cutoff, dh):
    """On a periodic sample wider than twice the cutoff, every row holds the sites of the
    infinite lattice within the cutoff (D_H = that count + the diagonal); 61, 124 and 235 are
    the densities of the benchmark's three cutoffs."""
    lat = olat.build_lattice(kind, L, t=-2.7, cutoff=cutoff, decay=DECAY)
    want = _count_infinite(kind, cutoff)
    assert np.all(np.asarray(lat.degree) == want)
    if dh is not None:
        assert want + 1 == dh
    # every bond is a distinct column (no image coincides) and H is real symmetric
    assert lat.H.nnz == lat.n * (want + 1) - np.count_nonzero(lat.H.diagonal() == 0)
    assert abs(lat.H - lat.H.T).max() < 1e-13   # distances from positions up to ~70 apart, to rounding


def _bloch_honeycomb(k, cutoff, t, decay):
    h = np.zeros((2, 2), np.complex128)
    R = int(cutoff) + 2
    for s, sp_ in itertools.product((0, 1), (0, 1)):
        for m, q in itertools.product(range(-R, R + 1), range(-R, R + 1)):
            d = m * A1 + q * A2 + (sp_ - s) * np.array([1.0, 0, 0])
            r = np.linalg.norm(d)
            if 1e-9 < r <= cutoff:
                h[s, sp_] += _t(r, t, decay) * np.exp(1j * (k @ d))
    return h


@pytest.mark.parametrize("L,cutoff", [((6, 5, 1), 3.3), ((3, 4, 1), 4.1), ((9, 7, 1), 2.1)])
def test_honeycomb_bloch_states(L, cutoff):
    """Bloch's theorem on the periodic long-range honeycomb: psi(c, s) = u_s e^{i k.r} with k on
    the sample's reciprocal grid satisfies H psi = (h(k) u)_s e^{i k.r}, h(k) the 2 x 2 lattice
    sum over all bond vectors d within the cutoff of t(|d|) e^{i k.d}.  Holds also when images
    of one site coincide (small samples)."""
    t = -2.7
    lat = olat.build_lattice(olat.HONEYCOMB, L, t=t, cutoff=cutoff, decay=0.7)
    Lx, Ly, _ = L
    # reciprocal vectors: b_i . a_j = 2 pi delta_ij (in the plane)
    Am = np.array([A1[:2], A2[:2]])
    B = 2 * np.pi * np.linalg.inv(Am).T
    full = np.arange(lat.n_full)
    pos = olat.site_positions(olat.HONEYCOMB, lat.L, full)
    s = full % 2
    rng = np.random.default_rng(1)
    for mx, my in [(0, 0), (1, 2), (Lx - 1, 1), (2, Ly - 1)]:
        k = np.zeros(3)
        k[:2] = mx / Lx * B[0] + my / Ly * B[1]
        u = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        psi = u[s] * np.exp(1j * (pos @ k))
        want = (_bloch_honeycomb(k, cutoff, t, 0.7) @ u)[s] * np.exp(1j * (pos @ k))
        assert np.max(np.abs(lat.H @ psi - want)) < 1e-12


@pytest.mark.parametrize("L", [(7, 5, 1), (2, 3, 1)])
def test_square_plane_waves(L):
    """Square lattice: e^{i k.r} has E(k) = sum over lattice vectors 0 < |R| <= cutoff of t(|R|) cos(k.R)."""
    t, cutoff, decay = 1.1, 2.9, 0.6
    lat = olat.build_lattice(olat.SQUARE, L, t=t, cutoff=cutoff, decay=decay)
    Lx, Ly, _ = L
    x, y = np.arange(lat.n) % Lx, np.arange(lat.n) // Lx
    for mx, my in [(0, 0), (1, 1), (3 % Lx, 2 % Ly)]:
        kx, ky = 2 * np.pi * mx / Lx, 2 * np.pi * my / Ly
        v = np.exp(1j * (kx * x + ky * y))
        E = 0.0
        for a, b in itertools.product(range(-4, 5), range(-4, 5)):
            r = math.hypot(a, b)
            if 0 < r <= cutoff:
                E += _t(r, t, decay) * math.cos(kx * a + ky * b)
        assert np.max(np.abs(lat.H @ v - E * v)) < 1e-12


def test_vacancies_restrict_the_clean_hamiltonian_and_bounds_hold():
    spec = dict(t=-2.7, W=1.5, seed=9, cutoff=3.1, decay=DECAY)
    full = olat.build_lattice(olat.HONEYCOMB, (8, 7, 1), **spec)
    vac = olat.build_lattice(olat.HONEYCOMB, (8, 7, 1), vacancy_frac=0.08, **spec)
    keep = np.flatnonzero(vac.active)
    assert 0 < keep.size < full.n
    sub = full.H[keep][:, keep]
    assert abs(sub - vac.H).max() < 1e-15
    ev = np.linalg.eigvalsh(vac.H.toarray())
    assert vac.E_min <= ev[0] and ev[-1] <= vac.E_max
    # open boundaries keep fewer bonds than the periodic sample
    op = olat.build_lattice(olat.HONEYCOMB, (8, 7, 1), pbc=(0, 0, 1), **spec)
    assert op.H.nnz < full.H.nnz and isinstance(op.H, sp.csr_matrix)


def test_long_range_needs_a_decay_length():
    with pytest.raises(ValueError):
        olat.build_lattice(olat.SQUARE, (4, 4, 1), t=1.0, cutoff=2.0, decay=0.0)


@pytest.mark.parametrize("kind,L,pbc", [(olat.HONEYCOMB, (5, 4, 1), (1, 1, 1)), (olat.HONEYCOMB, (6, 3, 1), (0, 1, 1)),
                                        (olat.SQUARE, (5, 6, 1), (1, 0, 1)), (olat.CUBIC, (3, 4, 3), (1, 1, 1))])
def test_current_operator_at_cutoff_one_is_the_nearest_neighbour_one(kind, L, pbc):
    from oracle import conductivity as oec
    nn = olat.build_lattice(kind, L, t=-1.3, W=0.7, seed=5, pbc=pbc)
    lr = olat.build_lattice(kind, L, t=-1.3, W=0.7, seed=5, pbc=pbc, cutoff=1.2, decay=0.5)
    for a in range(3 if kind == olat.CUBIC else 2):
        assert abs(oec.current_operator(nn, a) - oec.current_operator(lr, a)).max() < 4e-15


@pytest.mark.parametrize("L,cutoff", [((6, 5, 1), 3.3), ((3, 4, 1), 4.1)])
def test_current_operator_is_the_band_velocity(L, cutoff):
    """J_a = i[H, P_a] on Bloch states: J psi = (-dh/dk_a u)_s e^{i k.r}, with
    dh/dk_a = sum_d t(|d|) i d_a e^{i k.d} the derivative of the lattice sum h(k)."""
    from oracle import conductivity as oec
    t, decay = -2.7, 0.7
    lat = olat.build_lattice(olat.HONEYCOMB, L, t=t, cutoff=cutoff, decay=decay)
    Lx, Ly, _ = L
    Am = np.array([A1[:2], A2[:2]])
    B = 2 * np.pi * np.linalg.inv(Am).T
    full = np.arange(lat.n_full)
    pos = olat.site_positions(olat.HONEYCOMB, lat.L, full)
    s = full % 2
    rng = np.random.default_rng(2)
    R = int(cutoff) + 2
    for mx, my in [(1, 2), (Lx - 1, 1), (0, 0)]:
        k = np.zeros(3)
        k[:2] = mx / Lx * B[0] + my / Ly * B[1]
        for a in (0, 1):
            dh = np.zeros((2, 2), np.complex128)
            for s0, s1 in itertools.product((0, 1), (0, 1)):
                for m, q in itertools.product(range(-R, R + 1), range(-R, R + 1)):
                    d = m * A1 + q * A2 + (s1 - s0) * np.array([1.0, 0, 0])
                    r = np.linalg.norm(d)
                    if 1e-9 < r <= cutoff:
                        dh[s0, s1] += _t(r, t, decay) * 1j * d[a] * np.exp(1j * (k @ d))
            u = rng.standard_normal(2) + 1j * rng.standard_normal(2)
            psi = u[s] * np.exp(1j * (pos @ k))
            want = (-(dh @ u))[s] * np.exp(1j * (pos @ k))
            J = oec.current_operator(lat, a)
            assert np.max(np.abs(J @ psi - want)) < 1e-12
            assert abs(J - J.conj().T).max() < 1e-13
