"""Pins of the oracle's honeycomb window (a piece of a large periodic lattice with the whole
lattice's disorder and spectral bounds), used to check LDOS moments of lattices too large for
the oracle on sampled sites.  The window must reproduce the whole lattice's on-site energies at
the same global sites and its site moments <r|T_n(H~)|r> for n up to the radius, and must
differ once a walk from the site can reach the window's edge and return (so the check is not
vacuous)."""
import numpy as np

from oracle import lattice as olat, propagate as oprop


def unit(n, i):
    v = np.zeros(n, np.complex128)
    v[i] = 1.0
    return v


def test_window_reproduces_whole_lattice_moments_inside_the_light_cone():
    L, t, W, seed, R = (40, 36), -2.7, 1.0, 5, 8
    ol = olat.build_lattice(olat.HONEYCOMB, L + (1,), t=t, W=W, seed=seed)
    for center in ((0, 0), (17, 35), (39, 20)):       # two of them wrap around both directions
        wl, ia, ib, full = olat.honeycomb_window(L, center, R, t, W, seed, ol.E_min, ol.E_max)
        assert np.array_equal(wl.V, ol.V[full])
        assert (wl.H0, wl.half_width) == (ol.H0, ol.half_width)
        for local, s in ((ia, 0), (ib, 1)):
            g = 2 * (center[1] * L[0] + center[0]) + s
            assert full[local] == g
            mw = oprop.moments(wl, unit(wl.n, local), unit(wl.n, local), 6 * R)
            mf = oprop.moments(ol, unit(ol.n, g), unit(ol.n, g), 6 * R)
            assert np.max(np.abs(mw[:R + 1] - mf[:R + 1])) < 1e-13
            # once a walk can reach the window's edge and come back, the edge is felt
            assert np.max(np.abs(mw[4 * R + 4:] - mf[4 * R + 4:])) > 1e-6


def test_window_rejects_a_radius_that_wraps():
    import pytest
    with pytest.raises(ValueError):
        olat.honeycomb_window((10, 10), (0, 0), 5, -2.7, 0.0, 1, -8.1, 8.1)
