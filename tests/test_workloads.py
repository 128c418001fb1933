"""The seeded synthetic input recipe: sizes, seeds and request streams of the workloads module.

The module is shared by the tests, the oracle runs and the benchmark, and holds only parameters:
these checks pin the sizes the measurements quote (the 8,388,608-site benchmark lattice, the
1,015,021,568-site largest lattice, the 4,763,200-site dense samples that stand in for the paper's
twisted bilayer), the midpoint energy grid, the LDOS site lists and the serving stream's
distributions, and that the module imports neither the oracle nor the library."""
import math

import numpy as np

import workloads as wl


def test_lattice_sizes_of_the_workloads():
    assert wl.GRAPHENE_2048.lattice.n_full == 8_388_608
    assert wl.GRAPHENE_22528.lattice.n_full == 1_015_021_568
    assert wl.GRAPHENE_4096_VAC.lattice.n_full == 33_554_432
    assert wl.SQUARE_64.lattice.n_full == 4096
    for dh in (61, 124, 235):
        w = wl.dense_honeycomb(dh)
        assert w.lattice.n_full == 4_763_200  # the paper's atom count
        assert w.lattice.cutoff == wl.DENSE_CUTOFFS[dh] and w.lattice.decay == wl.DENSE_DECAY
    assert wl.cubic(3, 4, 5).n_full == 60
    assert wl.GRAPHENE_2048.n_states == 8 and wl.GRAPHENE_2048.n_moments == 4096
    assert wl.GRAPHENE_22528.n_states == 4 and wl.GRAPHENE_22528.n_moments == 8192
    assert wl.GRAPHENE_4096_VAC.lattice.vacancy_frac == 0.01 and wl.GRAPHENE_4096_VAC.n_steps == 2048


def test_seeds_and_disorder_widths():
    assert wl.LATTICE_SEED == 0x7B1A5 and wl.REQUEST_SEED == 0xC0FFEE
    # W is the full width of the uniform on-site distribution: V in [-W/2, W/2]
    assert wl.SQUARE_64.lattice.W == 1.0                 # V in [-0.5, 0.5]
    assert wl.GRAPHENE_4096_VAC.lattice.W == 2.0         # V in [-1, 1] eV
    assert wl.GRAPHENE_22528.lattice.W == 1.0            # V in [-0.5, 0.5] eV
    assert wl.GRAPHENE_2048.lattice.W == 0.0


def test_midpoint_energy_grid():
    E = wl.uniform_energy_grid(8, -1.0, 1.0)
    assert np.allclose(E, -1.0 + (2 * np.arange(8) + 1) / 8)
    assert np.allclose(np.diff(E), 0.25) and np.allclose(E + E[::-1], 0.0)
    assert E.min() > -1.0 and E.max() < 1.0


def test_ldos_sites_are_distinct_sorted_and_reproducible():
    a = wl.ldos_sites(1000, 32, seed=7)
    b = wl.ldos_sites(1000, 32, seed=7)
    assert a.dtype == np.int64 and np.array_equal(a, b)
    assert len(np.unique(a)) == 32 and np.all(np.diff(a) > 0)
    assert a.min() >= 0 and a.max() < 1000
    assert not np.array_equal(a, wl.ldos_sites(1000, 32, seed=8))


def test_serving_stream_distributions():
    rate = 4.0
    reqs = wl.serving_stream(512, rate)
    again = wl.serving_stream(512, rate)
    assert [(r.arrival_s, r.n_moments, r.n_states, r.lattice) for r in reqs] == \
           [(r.arrival_s, r.n_moments, r.n_states, r.lattice) for r in again]
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * rate - 1.0) < 0.15          # Poisson arrivals at the given rate
    kinds = {r.lattice.kind for r in reqs}
    assert kinds == {wl.SQUARE, wl.HONEYCOMB, wl.CUBIC}
    for r in reqs:
        n = r.lattice.n_full
        # L is rounded from a log-uniform target in [2^12, 2^24]: a cube's edge moves the count most
        assert 2 ** 12 * 0.85 <= n <= 2 ** 24 * 1.15, n
        assert r.n_moments % 8 == 0 and 256 <= r.n_moments <= 8192
        assert 0.0 <= r.lattice.W <= 2.0 and r.lattice.t == 1.0
        if r.quantity == "ldos":
            assert r.n_states == 32 and len(np.unique(r.sites)) == 32
            assert r.sites.min() >= 0 and r.sites.max() < n
        else:
            assert r.quantity == "dos" and r.sites is None and 1 <= r.n_states <= 16
    logs = np.log2([r.lattice.n_full for r in reqs])
    assert abs(np.median(logs) - 18.0) < 1.0             # log-uniform over 12..24
    assert 0.35 < np.mean([r.quantity == "ldos" for r in reqs]) < 0.65


def test_serving_stream_size_cap():
    reqs = wl.serving_stream(64, 1.0, log2_max=20)
    assert max(r.lattice.n_full for r in reqs) <= 2 ** 20 * 1.15


def test_module_holds_no_method_code():
    src = open(wl.__file__).read()
    assert "import oracle" not in src and "from oracle" not in src
    assert "paper_2510_17432_gb300" not in src
    assert math.isclose(wl.DENSE_DECAY, 0.3187)
