"""Chebyshev recurrence, moments and time propagation (FP64), written from Sec. II.A.

Definitions followed, in the paper's notation:
* Chebyshev states  phi_0 = psi, phi_1 = H~ psi, phi_{n+1} = 2 H~ phi_n - phi_{n-1}
  (App. B, Eq. cheb_relation), H~ = (H - H0)/|H|.
* Moments  m_n = <psi_1| T_n(H~) |psi_2>  (Sec. II.A, moment-based implementation).
* Sequential propagation (Sec. II.A):
      |psi(t_j)> = exp(-i H0 tau) sum_{n<N(tau~)} c_n(tau~) T_n(H~) |psi(t_{j-1})>,
  t_j = j tau, tau = tau~/|H|; C(t_j) = <psi|psi(t_j)> (Sec. III).  The paper drops the
  exp(-i H0 t) factor (its spectra are centred); it is kept here and equals 1 when H0 = 0.
* Moment-based concurrent form (Sec. III, DOS-Concurrent-M):
      C(t_j) = exp(-i H0 t_j) sum_{n<N(j tau~)} c_n(j tau~) m_n.
* State-based concurrent form with time blocks of b steps (Sec. II.A Eq. TE, Sec. II.B):
  from chi = psi(t_{kb}), psi(t_{kb+j}) = exp(-i H0 j tau) sum_{n<N(j tau~)} c_n(j tau~) T_n chi.
* Cost-halving for psi_1 = psi_2 (Sec. II.A, Eqs. cheby_prod and cheby-moment).  The
  printed Eq. cheby-moment omits a factor 2 that Eq. cheby_prod requires; the reading
  used here is m_{2k} = 2<phi_k|phi_k> - m_0 and m_{2k+1} = 2<phi_{k+1}|phi_k> - m_1.

Every propagation counts its kernel calls in an OpCounter so that Tab. I can be
checked: one `amxsy` per Chebyshev term generated (T_0 included, as Tab. I counts
t~_tot R(tau~) = N_t N(tau~) per sequential run), one `axpy` per term accumulated
into a state, one `dot` per inner product producing an output value.

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .bessel import cheb_coefficients, truncation_order
from .lattice import Lattice, rescaled_apply
from .philox import draw_u32, STREAM_PHASE


@dataclass
class OpCounter:
    amxsy: int = 0
    axpy: int = 0
    dot: int = 0


def random_phase_states(lat: Lattice, state_seed: int, n_states: int) -> np.ndarray:
    """[S, n_active] complex128 random-phase states psi_i = exp(i theta_i)/sqrt(N_active).

    theta_i = 2 pi u / 2^32 with u the phase-stream Philox draw of the full site index i
    and state s (counter = (i, stream 2, s)).  Normalised so that <psi|psi> = 1."""
    full_idx = np.flatnonzero(lat.active).astype(np.uint64)
    out = np.empty((n_states, full_idx.size), dtype=np.complex128)
    norm = 1.0 / np.sqrt(float(full_idx.size))
    for s in range(n_states):
        u = draw_u32(state_seed, full_idx, STREAM_PHASE, s).astype(np.float64)
        theta = 2.0 * np.pi * (u / 4294967296.0)
        out[s] = (np.cos(theta) + 1j * np.sin(theta)) * norm
    return out


def site_states(lat: Lattice, sites) -> np.ndarray:
    """LDOS states |r> (Sec. III): unit vectors on the given compact site indices."""
    sites = np.asarray(sites, dtype=np.int64)
    out = np.zeros((sites.size, lat.n), dtype=np.complex128)
    out[np.arange(sites.size), sites] = 1.0
    return out


def chebyshev_states(lat: Lattice, psi: np.ndarray, n_terms: int, ops: OpCounter | None = None):
    """Yield phi_n = T_n(H~) psi for n = 0..n_terms-1."""
    prev, cur = None, psi.astype(np.complex128)
    for n in range(n_terms):
        if n == 0:
            nxt = cur
        elif n == 1:
            nxt = rescaled_apply(lat, cur)
        else:
            nxt = 2.0 * rescaled_apply(lat, cur) - prev
        if ops is not None:
            ops.amxsy += 1
        if n >= 1:
            prev, cur = cur, nxt
        yield nxt


def moments(lat: Lattice, bra: np.ndarray, ket: np.ndarray, n_moments: int,
            ops: OpCounter | None = None) -> np.ndarray:
    """m_n = <bra| T_n(H~) |ket>, n = 0..n_moments-1 (plain definition)."""
    out = np.empty(n_moments, dtype=np.complex128)
    for n, phi in enumerate(chebyshev_states(lat, ket, n_moments, ops)):
        out[n] = np.vdot(bra, phi)
        if ops is not None:
            ops.dot += 1
    return out


def moments_doubling(lat: Lattice, psi: np.ndarray, n_moments: int,
                     ops: OpCounter | None = None) -> np.ndarray:
    """Moments of <psi|T_n|psi> from phi_0..phi_{M/2} with the product identity
    2 T_m T_n = T_{m+n} + T_{|m-n|} (Eq. cheby_prod):
        m_{2k} = 2 <phi_k|phi_k> - m_0,   m_{2k+1} = 2 <phi_{k+1}|phi_k> - m_1."""
    if n_moments % 2:
        raise ValueError("n_moments must be even")
    half = n_moments // 2
    phis = []
    for phi in chebyshev_states(lat, psi, half + 1, ops):
        phis.append(phi)
    m = np.empty(n_moments, dtype=np.complex128)
    m0 = np.vdot(psi, psi)
    m1 = np.vdot(psi, phis[1])
    for k in range(half):
        m[2 * k] = 2.0 * np.vdot(phis[k], phis[k]) - m0
        m[2 * k + 1] = 2.0 * np.vdot(phis[k + 1], phis[k]) - m1
        if ops is not None:
            ops.dot += 2
    m[0], m[1] = m0, m1
    return m


def evolve_step(lat: Lattice, psi: np.ndarray, tau: float, ops: OpCounter | None = None) -> np.ndarray:
    """exp(-i H tau_phys) psi with tau = tau~ (rescaled), Chebyshev series truncated at N(tau~)."""
    n_terms = truncation_order(abs(tau))
    c = cheb_coefficients(tau, n_terms)
    out = np.zeros_like(psi, dtype=np.complex128)
    for n, phi in enumerate(chebyshev_states(lat, psi, n_terms, ops)):
        out += c[n] * phi
        if ops is not None:
            ops.axpy += 1
    return np.exp(-1j * lat.H0 * tau / lat.half_width) * out


def correlation_sequential(lat: Lattice, psi: np.ndarray, n_steps: int, tau: float = np.pi,
                           ops: OpCounter | None = None, return_norms: bool = False):
    """C(t_j) = <psi|psi(t_j)>, j = 0..n_steps, by step-by-step propagation (DOS-Sequential)."""
    C = np.empty(n_steps + 1, dtype=np.complex128)
    norms = np.empty(n_steps + 1)
    cur = psi.astype(np.complex128)
    C[0] = np.vdot(psi, cur)
    norms[0] = np.linalg.norm(cur)
    for j in range(1, n_steps + 1):
        cur = evolve_step(lat, cur, tau, ops)
        C[j] = np.vdot(psi, cur)
        norms[j] = np.linalg.norm(cur)
        if ops is not None:
            ops.dot += 1
    return (C, norms) if return_norms else C


def correlation_from_moments(mu: np.ndarray, n_steps: int, tau: float, shift: float) -> np.ndarray:
    """Moment-based concurrent reconstruction C(t_j) = exp(-i shift j tau~) sum_{n<N(j tau~)} c_n(j tau~) m_n.

    `shift` = H0/|H| so that exp(-i H0 t_j) = exp(-i shift * j tau~)."""
    C = np.empty(n_steps + 1, dtype=np.complex128)
    C[0] = mu[0]
    for j in range(1, n_steps + 1):
        tj = j * tau
        nj = truncation_order(abs(tj))
        if nj > mu.size:
            raise ValueError(f"step {j} needs {nj} moments, have {mu.size}")
        c = cheb_coefficients(tj, nj)
        C[j] = np.exp(-1j * shift * tj) * np.dot(c, mu[:nj])
    return C


def propagate_state_blocks(lat: Lattice, psi: np.ndarray, n_steps: int, b: int, tau: float = np.pi,
                           ops: OpCounter | None = None):
    """State-based concurrent propagation in time blocks of b steps.

    Returns (C, states) with C[j] = <psi|psi(t_j)> and states[j] = psi(t_j), j = 0..n_steps."""
    shift = lat.H0 / lat.half_width
    states = np.empty((n_steps + 1, psi.size), dtype=np.complex128)
    states[0] = psi
    C = np.empty(n_steps + 1, dtype=np.complex128)
    C[0] = np.vdot(psi, psi)
    start = 0
    while start < n_steps:
        bb = min(b, n_steps - start)
        n_per = [truncation_order(j * tau) for j in range(1, bb + 1)]
        coeff = [cheb_coefficients(j * tau, n_per[j - 1]) for j in range(1, bb + 1)]
        acc = np.zeros((bb, psi.size), dtype=np.complex128)
        for n, phi in enumerate(chebyshev_states(lat, states[start], max(n_per), ops)):
            for j in range(bb):
                if n < n_per[j]:
                    acc[j] += coeff[j][n] * phi
                    if ops is not None:
                        ops.axpy += 1
        for j in range(bb):
            states[start + j + 1] = np.exp(-1j * shift * (j + 1) * tau) * acc[j]
            C[start + j + 1] = np.vdot(psi, states[start + j + 1])
            if ops is not None:
                ops.dot += 1
        start += bb
    return C, states


def correlation_backward(lat: Lattice, psi: np.ndarray, n_steps: int, tau: float = np.pi) -> np.ndarray:
    """C(-t_j) by propagating with the negative step (coefficients c_n(-tau~) = 2 i^n J_n(tau~))."""
    return correlation_sequential(lat, psi, n_steps, -tau)
