"""Seeded synthetic workload descriptors shared by the tests, the oracle runs and bench.py.

This module holds only sizes, seeds and parameter choices: no arithmetic of the
method lives here.  Every random number the method draws (on-site disorder,
vacancies, random phases) is drawn by each side from the counter-based
Philox4x32-10 generator keyed by the seeds below, so this module never produces
an input array itself.  The only arrays it hands out are request parameters
(energy grids, LDOS site lists) built with a seeded numpy generator or plain
linspace, which are inputs of the method, not results of it.

Lattice kinds follow the tight-binding models of the paper's test systems
(nearest-neighbour graphene, Fig. 1; a square lattice and a simple-cubic lattice as
further regular stencils).  The paper's own primary test system (twisted bilayer
graphene, Sec. II.B) is not reproducible without its geometry; honeycomb
lattices stand in for it, with long-range hopping where the density D_H matters.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

SQUARE, HONEYCOMB, CUBIC = 0, 1, 2
KIND_NAMES = {SQUARE: "square", HONEYCOMB: "honeycomb", CUBIC: "cubic"}
COORDINATION = {SQUARE: 4, HONEYCOMB: 3, CUBIC: 6}

PATH_AUTO, PATH_STENCIL, PATH_CSR = 0, 1, 2

C64, C128 = 0, 1  # complex64 states with FP64 accumulation / complex128 states

LATTICE_SEED = 0x7B1A5
REQUEST_SEED = 0xC0FFEE


@dataclass(frozen=True)
class LatticeSpec:
    kind: int
    L: tuple  # (Lx, Ly, Lz); unused trailing entries are 1
    t: float = 1.0
    W: float = 0.0
    vacancy_frac: float = 0.0
    seed: int = LATTICE_SEED
    pbc: tuple = (1, 1, 1)
    path: int = PATH_AUTO
    cutoff: float = 0.0       # long-range hopping radius (0: nearest neighbours)
    decay: float = 0.0        # decay length of t(r) = t exp(-(r - 1)/decay)

    @property
    def n_full(self) -> int:
        Lx, Ly, Lz = self.L
        if self.kind == HONEYCOMB:
            return 2 * Lx * Ly
        if self.kind == SQUARE:
            return Lx * Ly
        return Lx * Ly * Lz


@dataclass(frozen=True)
class Workload:
    name: str
    lattice: LatticeSpec
    n_states: int
    n_moments: int
    precision: int
    state_seed: int = 1
    n_steps: int = 0          # time steps N_t for correlation requests
    n_energies: int = 0
    description: str = ""


def square(Lx, Ly, **kw) -> LatticeSpec:
    return LatticeSpec(SQUARE, (Lx, Ly, 1), **kw)


def honeycomb(Lx, Ly, **kw) -> LatticeSpec:
    return LatticeSpec(HONEYCOMB, (Lx, Ly, 1), **kw)


def cubic(Lx, Ly, Lz, **kw) -> LatticeSpec:
    return LatticeSpec(CUBIC, (Lx, Ly, Lz), **kw)


# The five workloads of the benchmark description, named by what they are.
SQUARE_64 = Workload(
    "square64x64_W1_c128_S1_M1024",
    square(64, 64, t=1.0, W=1.0),
    n_states=1, n_moments=1024, precision=C128, n_steps=295, n_energies=1024,
    description="square 64x64 PBC, t=1, V in [-0.5,0.5], complex128, 1 state, 1024 moments, DOS on 1024 energies")

GRAPHENE_2048 = Workload(
    "honeycomb2048x2048_S8_M4096",
    honeycomb(2048, 2048, t=-2.7, W=0.0),
    n_states=8, n_moments=4096, precision=C64, n_steps=1254, n_energies=8192,
    description="graphene 2048x2048 cells (8,388,608 sites), t=-2.7 eV, clean, complex64 + FP64 "
                "moment accumulation, 8 random-phase states, 4096 moments, Jackson DOS on 8192 energies")

GRAPHENE_4096_VAC = Workload(
    "honeycomb4096x4096_vac1pct_W2_Nt2048",
    honeycomb(4096, 4096, t=-2.7, W=2.0, vacancy_frac=0.01, path=PATH_CSR),
    n_states=1, n_moments=0, precision=C64, n_steps=2048, n_energies=64,
    description="graphene 4096x4096 cells, 1% vacancies (CSR path), V in [-1,1] eV, "
                "tau~=pi, 2048 steps, state-based blocks")

GRAPHENE_22528 = Workload(
    "honeycomb22528x22528_W1_S4_M8192",
    honeycomb(22528, 22528, t=-2.7, W=1.0),
    n_states=4, n_moments=8192, precision=C64, n_energies=2048,
    description="graphene 22528x22528 cells (1,015,021,568 sites), V in [-0.5,0.5] eV, stencil, "
                "complex64, 4 states, 8192 moments")


# Dense Hamiltonians standing in for the paper's 4,763,200-atom twisted bilayer graphene, whose
# density D_H it varies over 60, 120 and 230 (Sec. IV): a honeycomb sample of the same number of
# sites with every neighbour within the cutoff bonded, t(r) = t exp(-(r - 1)/decay), decay
# 0.3187 nearest-neighbour distances (0.184 lattice constants, the decay of the usual pz model
# of graphene bilayers).  Cutoffs 5.1, 7.1 and 9.7 give D_H = 61, 124 and 235 (taps + diagonal).
DENSE_DECAY = 0.3187
DENSE_CUTOFFS = {61: 5.1, 124: 7.1, 235: 9.7}


def dense_honeycomb(dh: int, n_states: int = 2, n_steps: int = 4096, L=(1832, 1300)) -> Workload:
    cutoff = DENSE_CUTOFFS[dh]
    Lx, Ly = L
    return Workload(
        f"honeycomb{Lx}x{Ly}_DH{dh}_S{n_states}_Nt{n_steps}",
        honeycomb(Lx, Ly, t=-2.7, W=0.0, cutoff=cutoff, decay=DENSE_DECAY),
        n_states=n_states, n_moments=0, precision=C64, n_steps=n_steps, n_energies=2048,
        description=f"honeycomb {Lx}x{Ly} cells ({2 * Lx * Ly} sites), long-range hopping within {cutoff} "
                    f"(D_H = {dh}), complex64, {n_states} states, DOS over N_t = {n_steps} steps of tau~ = pi")


def uniform_energy_grid(n: int, lo: float, hi: float) -> np.ndarray:
    """Midpoint grid of n energies on [lo, hi] (the request's energy samples)."""
    k = np.arange(n, dtype=np.float64)
    return lo + (hi - lo) * (k + 0.5) / n


def ldos_sites(n_sites_total: int, count: int, seed: int = REQUEST_SEED) -> np.ndarray:
    """Distinct site indices for LDOS requests, drawn with a seeded numpy generator."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_sites_total, size=count, replace=False)).astype(np.int64)


@dataclass
class ServingRequest:
    arrival_s: float
    lattice: LatticeSpec
    n_moments: int
    n_states: int
    quantity: str             # "dos" or "ldos"
    sites: np.ndarray | None = None


def serving_stream(n_requests: int, rate_per_s: float, seed: int = REQUEST_SEED,
                   log2_min: int = 12, log2_max: int = 24,
                   m_min: int = 256, m_max: int = 8192, s_max: int = 16,
                   ldos_count: int = 32):
    """Poisson-arrival request stream: lattice kind uniform over square/honeycomb/cubic,
    site count log-uniform in [2^log2_min, 2^log2_max], W uniform in [0, 2]t, moments
    uniform in [m_min, m_max] (rounded to a multiple of 8), 1..s_max states, DOS or LDOS
    at ldos_count sites."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        kind = int(rng.integers(0, 3))
        n_target = 2.0 ** rng.uniform(log2_min, log2_max)
        if kind == SQUARE:
            L = max(4, int(round(math.sqrt(n_target))))
            spec = square(L, L)
        elif kind == HONEYCOMB:
            L = max(4, int(round(math.sqrt(n_target / 2))))
            spec = honeycomb(L, L)
        else:
            L = max(4, int(round(n_target ** (1.0 / 3.0))))
            spec = cubic(L, L, L)
        tval = 1.0
        W = float(rng.uniform(0.0, 2.0)) * tval
        spec = replace(spec, t=tval, W=W, seed=int(rng.integers(1, 2**31)))
        M = int(rng.integers(m_min, m_max + 1)) // 8 * 8
        quantity = "ldos" if rng.random() < 0.5 else "dos"
        if quantity == "ldos":
            sites = ldos_sites(spec.n_full, ldos_count, seed=int(rng.integers(1, 2**31)))
            S = ldos_count
        else:
            sites = None
            S = int(rng.integers(1, s_max + 1))
        out.append(ServingRequest(t, spec, M, S, quantity, sites))
    return out
