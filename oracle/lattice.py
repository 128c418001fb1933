"""Tight-binding lattices and Hamiltonians for the FP64 oracle.

The paper's operator is a sparse tight-binding Hamiltonian H with nearest-neighbour
hopping t and on-site terms (Sec. II.B defines its density D_H as the mean number
of non-zeros per row; Fig. 1 uses nearest-neighbour graphene).  The paper prints no
lattice code, so the site numbering, neighbour order, disorder and vacancy rules
below are this library's own convention, fixed bit for bit by golden files:

* square  Lx x Ly:  site i = y*Lx + x; neighbours (x+1,y), (x-1,y), (x,y+1), (x,y-1).
* honeycomb Lx x Ly cells: site i = 2*(y*Lx + x) + s, s=0 (A) or 1 (B).
  A(x,y) bonds to B(x,y), B(x-1,y), B(x,y-1);  B(x,y) bonds to A(x,y), A(x+1,y), A(x,y+1).
* simple cubic Lx x Ly x Lz: site i = (z*Ly + y)*Lx + x; neighbours +-x, +-y, +-z.
Periodic directions wrap by modulo; open directions drop the bond.
H_ij = t for every bond (bonds that coincide under wrapping add up), H_ii = V_i.

Anderson disorder: V_i = W * ((u >> 8) * 2^-24 - 1/2), u = Philox draw of site i in the
disorder stream, so V_i is uniform on [-W/2, W/2).  Vacancies: site i is removed when
its vacancy-stream draw u < floor(p * 2^32).  Active sites are renumbered in order.

Spectral bounds (the paper takes H0 and |H| "typically" from Lanczos, Sec. II.A; the
reading used here is Gershgorin, which never underestimates):
    E_max = max_i (V_i + deg_i |t|),  E_min = min_i (V_i - deg_i |t|)
    H0 = (E_max + E_min) / 2,  |H| = (1 + 0.01) (E_max - E_min) / 2.

Long-range hopping (cutoff > 0).  The paper's test system is a dense Hamiltonian whose
density D_H (non-zeros per row, Sec. II.B) it varies from 60 to 230 (Sec. IV); its
geometry is not available, so a lattice of the same kinds stands in: every pair of sites
whose distance r (in units of the nearest-neighbour distance, positions below) satisfies
0 < r <= cutoff is bonded with t(r) = t exp(-(r - 1)/decay), t(1) = t.  With periodic
boundaries H_ij sums t(|r_j + R - r_i|) over every period vector R of the sample that
brings the pair within the cutoff (images add up, as coinciding bonds do above); open
directions take R = 0 only.  Gershgorin then uses sum_j |t| over all those bonds.
Positions: square (x, y, 0); cubic (x, y, z); honeycomb x a1 + y a2 + s (1, 0, 0) with
a1 = (3/2, sqrt3/2, 0), a2 = (3/2, -sqrt3/2, 0), so A(x,y)-B(x,y) has length 1.

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .philox import draw_u32, STREAM_DISORDER, STREAM_VACANCY

SQUARE, HONEYCOMB, CUBIC = 0, 1, 2
SQ3 = np.sqrt(3.0)
COORDINATION = {SQUARE: 4, HONEYCOMB: 3, CUBIC: 6}
BOUND_MARGIN = 0.01


def full_site_count(kind: int, L) -> int:
    Lx, Ly, Lz = L
    if kind == SQUARE:
        return Lx * Ly
    if kind == HONEYCOMB:
        return 2 * Lx * Ly
    if kind == CUBIC:
        return Lx * Ly * Lz
    raise ValueError(f"unknown lattice kind {kind}")


def _wrap(v, n, periodic):
    """Coordinate v in [-1, n] mapped into the box; -1 marks a dropped (open) bond."""
    if periodic:
        return np.mod(v, n), np.ones_like(v, dtype=bool)
    ok = (v >= 0) & (v < n)
    return np.where(ok, v, 0), ok


def neighbour_table(kind: int, L, pbc) -> np.ndarray:
    """int64 array [n_full, z] of neighbour site indices in the fixed neighbour order;
    -1 where an open boundary drops the bond."""
    Lx, Ly, Lz = L
    n = full_site_count(kind, L)
    i = np.arange(n, dtype=np.int64)
    cols = []
    if kind == SQUARE:
        x, y = i % Lx, i // Lx
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            xx, okx = _wrap(x + dx, Lx, pbc[0])
            yy, oky = _wrap(y + dy, Ly, pbc[1])
            cols.append(np.where(okx & oky, yy * Lx + xx, -1))
    elif kind == HONEYCOMB:
        s, c = i % 2, i // 2
        x, y = c % Lx, c // Lx
        # (dx, dy) to the partner cell for A (s=0) and for B (s=1)
        for (dxa, dya), (dxb, dyb) in (((0, 0), (0, 0)), ((-1, 0), (1, 0)), ((0, -1), (0, 1))):
            dx = np.where(s == 0, dxa, dxb)
            dy = np.where(s == 0, dya, dyb)
            xx, okx = _wrap(x + dx, Lx, pbc[0])
            yy, oky = _wrap(y + dy, Ly, pbc[1])
            cols.append(np.where(okx & oky, 2 * (yy * Lx + xx) + (1 - s), -1))
    elif kind == CUBIC:
        x, y, z = i % Lx, (i // Lx) % Ly, i // (Lx * Ly)
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            xx, okx = _wrap(x + dx, Lx, pbc[0])
            yy, oky = _wrap(y + dy, Ly, pbc[1])
            zz, okz = _wrap(z + dz, Lz, pbc[2])
            cols.append(np.where(okx & oky & okz, (zz * Ly + yy) * Lx + xx, -1))
    else:
        raise ValueError(f"unknown lattice kind {kind}")
    return np.stack(cols, axis=1).astype(np.int64)


def disorder_at(seed: int, W: float, full_idx) -> np.ndarray:
    """Anderson on-site energies V_i of the listed full site indices, uniform on [-W/2, W/2), FP64."""
    u = draw_u32(seed, np.asarray(full_idx, dtype=np.uint64), STREAM_DISORDER).astype(np.float64)
    frac = np.floor(u / 256.0) * 2.0 ** -24          # (u >> 8) * 2^-24, exact
    return W * (frac - 0.5)


def disorder_potential(seed: int, W: float, n_full: int) -> np.ndarray:
    """Anderson on-site energies V_i, uniform on [-W/2, W/2), FP64, by full site index."""
    return disorder_at(seed, W, np.arange(n_full, dtype=np.uint64))


def vacancy_threshold(p: float) -> int:
    return int(np.floor(np.float64(p) * 4294967296.0))


def vacancy_mask(seed: int, p: float, n_full: int) -> np.ndarray:
    """True where the site is removed."""
    if p <= 0.0:
        return np.zeros(n_full, dtype=bool)
    u = draw_u32(seed, np.arange(n_full, dtype=np.uint64), STREAM_VACANCY).astype(np.int64)
    return u < vacancy_threshold(p)


@dataclass
class Lattice:
    kind: int
    L: tuple
    pbc: tuple
    t: float
    W: float
    vacancy_frac: float
    seed: int
    n_full: int
    nbr_full: np.ndarray      # [n_full, z] full-index neighbours (-1 = none)
    active: np.ndarray        # [n_full] bool
    compact: np.ndarray       # [n_full] compact index or -1
    V: np.ndarray             # [n_active] FP64 on-site energies
    H: sp.csr_matrix          # [n_active, n_active] FP64
    degree: np.ndarray        # [n_active] bonds to active sites
    E_min: float
    E_max: float
    H0: float
    half_width: float
    cutoff: float = 0.0       # long-range hopping radius (0: nearest neighbours)
    decay: float = 0.0        # decay length of t(r)

    @property
    def n(self) -> int:
        return int(self.V.shape[0])


def site_positions(kind: int, L, full_idx) -> np.ndarray:
    """[len(full_idx), 3] positions of full sites (nearest-neighbour distance 1)."""
    Lx, Ly, Lz = L
    f = np.asarray(full_idx, dtype=np.int64)
    if kind == HONEYCOMB:
        s, c = f % 2, f // 2
        x, y = c % Lx, c // Lx
        return (x[:, None] * np.array([1.5, SQ3 / 2, 0.0]) + y[:, None] * np.array([1.5, -SQ3 / 2, 0.0])
                + s[:, None] * np.array([1.0, 0.0, 0.0]))
    if kind == CUBIC:
        return np.stack([f % Lx, (f // Lx) % Ly, f // (Lx * Ly)], axis=1).astype(np.float64)
    return np.stack([f % Lx, f // Lx, np.zeros(f.size)], axis=1).astype(np.float64)


def period_vectors(kind: int, L) -> list:
    """The sample's period vector along each of the three directions."""
    Lx, Ly, Lz = L
    if kind == HONEYCOMB:
        return [Lx * np.array([1.5, SQ3 / 2, 0.0]), Ly * np.array([1.5, -SQ3 / 2, 0.0]), np.zeros(3)]
    return [np.array([Lx, 0.0, 0.0]), np.array([0.0, Ly, 0.0]), np.array([0.0, 0.0, Lz if kind == CUBIC else 0.0])]


def long_range_bonds(kind: int, L, pbc, full_idx, t: float, cutoff: float, decay: float, with_disp: bool = False):
    """All bonds (i, j, t(r)) between the listed sites, by brute force over site pairs and
    period images: 0 < |r_j + R - r_i| <= cutoff.  Returns compact rows, columns, values (and,
    with_disp, the bond vectors r_j + R - r_i, [n_bonds, 3])."""
    dims = 3 if kind == CUBIC else 2
    pos = site_positions(kind, L, full_idx)[:, :dims]
    per = [v[:dims] for v in period_vectors(kind, L)]
    # r_j - r_i has fractional coordinates in (-1, 1) along the periods, so an image R = sum n_a
    # per_a can bring a pair within the cutoff only if |n_a| <= ceil(cutoff / h_a), h_a being the
    # sample's height across period a (its volume over the area of the other periods' face)
    vol = abs(np.linalg.det(np.array(per[:dims])))
    ranges = []
    for a in range(3):
        if a < dims and pbc[a]:
            others = [per[b] for b in range(dims) if b != a]
            face = np.linalg.norm(others[0]) if dims == 2 else np.linalg.norm(np.cross(others[0], others[1]))
            m = int(np.ceil(cutoff / (vol / face)))
            ranges.append(range(-m, m + 1))
        else:
            ranges.append(range(0, 1))
    rows, cols, vals, disp = [], [], [], []
    n = pos.shape[0]
    c2 = cutoff * cutoff
    for n0 in ranges[0]:
        for n1 in ranges[1]:
            for n2 in ranges[2]:
                R = n0 * per[0] + n1 * per[1] + (n2 * per[2] if dims == 3 else 0.0)
                for lo in range(0, n, 1024):
                    d2 = np.zeros((min(1024, n - lo), n))
                    for a in range(dims):
                        comp = pos[None, :, a] + R[a] - pos[lo:lo + 1024, None, a]
                        d2 += comp * comp
                    ii, jj = np.nonzero((d2 > 1e-18) & (d2 <= c2))
                    r = np.sqrt(d2[ii, jj])
                    rows.append(ii + lo)
                    cols.append(jj)
                    vals.append(t * np.exp(-(r - 1.0) / decay))
                    if with_disp:
                        dv = np.zeros((ii.size, 3))
                        for a in range(dims):
                            dv[:, a] = pos[jj, a] + R[a] - pos[ii + lo, a]
                        disp.append(dv)
    cat = lambda v, dt: np.concatenate(v).astype(dt) if v else np.zeros(0, dt)
    out = (cat(rows, np.int64), cat(cols, np.int64), cat(vals, np.float64))
    if with_disp:
        out = out + (np.concatenate(disp) if disp else np.zeros((0, 3)),)
    return out


def build_lattice(kind: int, L, t: float, W: float = 0.0, vacancy_frac: float = 0.0,
                  seed: int = 0, pbc=(1, 1, 1), cutoff: float = 0.0, decay: float = 0.0) -> Lattice:
    L = tuple(int(v) for v in L) + (1,) * (3 - len(L))
    pbc = tuple(bool(v) for v in pbc) + (True,) * (3 - len(pbc))
    n_full = full_site_count(kind, L)
    nbr = neighbour_table(kind, L, pbc)
    vac = vacancy_mask(seed, vacancy_frac, n_full)
    active = ~vac
    compact = np.full(n_full, -1, dtype=np.int64)
    compact[active] = np.arange(int(active.sum()), dtype=np.int64)
    V_full = disorder_potential(seed, W, n_full) if W != 0.0 else np.zeros(n_full)

    full_idx = np.flatnonzero(active)
    n = full_idx.size
    if cutoff > 0.0:
        if not decay > 0.0:
            raise ValueError("long-range hopping needs decay > 0")
        rows, cols, tv = long_range_bonds(kind, L, pbc, full_idx, float(t), float(cutoff), float(decay))
        nbr = None
    else:
        rows, cols = [], []
        for k in range(nbr.shape[1]):
            j = nbr[full_idx, k]
            keep = j >= 0
            keep[keep] &= active[j[keep]]
            rows.append(compact[full_idx[keep]])
            cols.append(compact[j[keep]])
        rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
        cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
        tv = np.full(rows.size, float(t))
    V = V_full[full_idx].astype(np.float64)
    hop = sp.coo_matrix((tv, (rows, cols)), shape=(n, n)).tocsr()
    H = (hop + sp.diags(V)).tocsr()
    H.sum_duplicates()
    degree = np.bincount(rows, minlength=n).astype(np.int64)
    if cutoff > 0.0:
        radius = np.bincount(rows, weights=np.abs(tv), minlength=n)   # sum of |t| over bonds
    else:
        radius = degree * abs(float(t))

    if n == 0:
        raise ValueError("lattice has no active sites")
    E_max = float(np.max(V + radius))
    E_min = float(np.min(V - radius))
    if not E_max > E_min:
        raise ValueError("degenerate spectrum: no hopping")
    H0 = (E_max + E_min) / 2.0
    half = (1.0 + BOUND_MARGIN) * (E_max - E_min) / 2.0
    return Lattice(kind, L, pbc, float(t), float(W), float(vacancy_frac), int(seed), n_full,
                   nbr, active, compact, V, H, degree, E_min, E_max, H0, half, float(cutoff), float(decay))


def honeycomb_window(L, center, radius: int, t: float, W: float, seed: int, E_min: float, E_max: float):
    """The cells of a periodic honeycomb lattice within `radius` cells of `center` = (x, y) in
    x and in y, as a lattice of their own: the global site numbering (for the disorder draw),
    nearest-neighbour bonds between window sites only, and the spectral bounds E_min, E_max of
    the WHOLE lattice (so that H~ = (H - H0)/|H| is the whole lattice's rescaling).

    A state supported on the centre cell reaches at most n cells in x and in y after n
    applications of H, so T_n(H~) applied to it, and its moments <r|T_n(H~)|r>, agree with the
    whole lattice's for n <= radius: a way to check any lattice, however large, on sampled sites.
    Returns (lattice, local index of A(center), local index of B(center), full index of every
    window site)."""
    Lx, Ly = int(L[0]), int(L[1])
    if 2 * radius + 1 > min(Lx, Ly):
        raise ValueError("window wraps onto itself")
    w = 2 * radius + 1
    dx, dy = np.meshgrid(np.arange(-radius, radius + 1), np.arange(-radius, radius + 1), indexing="xy")
    gx = (center[0] + dx.ravel()) % Lx
    gy = (center[1] + dy.ravel()) % Ly
    cells = w * w
    full = np.empty(2 * cells, dtype=np.int64)
    full[0::2] = 2 * (gy * Lx + gx)
    full[1::2] = full[0::2] + 1
    lx = dx.ravel() + radius
    ly = dy.ravel() + radius

    def cell(ix, iy):
        ok = (ix >= 0) & (ix < w) & (iy >= 0) & (iy < w)
        return np.where(ok, iy * w + ix, -1)

    a = 2 * np.arange(cells)
    rows, cols = [], []
    for ddx, ddy in ((0, 0), (-1, 0), (0, -1)):        # A(x,y) - B(x+ddx, y+ddy)
        c = cell(lx + ddx, ly + ddy)
        keep = c >= 0
        rows += [a[keep], 2 * c[keep] + 1]
        cols += [2 * c[keep] + 1, a[keep]]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    n = 2 * cells
    V = disorder_at(seed, W, full) if W != 0.0 else np.zeros(n)
    H = (sp.coo_matrix((np.full(rows.size, float(t)), (rows, cols)), shape=(n, n)).tocsr() + sp.diags(V)).tocsr()
    H.sum_duplicates()
    H0 = (E_max + E_min) / 2.0
    half = (1.0 + BOUND_MARGIN) * (E_max - E_min) / 2.0
    lat = Lattice(HONEYCOMB, (w, w, 1), (False, False, True), float(t), float(W), 0.0, int(seed), n,
                  None, np.ones(n, dtype=bool), np.arange(n, dtype=np.int64), V, H,
                  np.bincount(rows, minlength=n).astype(np.int64), float(E_min), float(E_max), H0, half)
    centre = radius * w + radius
    return lat, 2 * centre, 2 * centre + 1, full


def rescaled_apply(lat: Lattice, x: np.ndarray) -> np.ndarray:
    """H~ x with H~ = (H - H0) / |H| (Sec. II.A)."""
    return (lat.H @ x - lat.H0 * x) / lat.half_width
