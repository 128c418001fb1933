"""Thin ctypes binding of the C ABI declared in include/tbpm.h (argument marshalling only).

Every function keeps the C name and forwards to libtbpm.so; a negative status raises
TbpmError with the library's message.  Host buffers are numpy arrays; device buffers
are anything with a `data_ptr()` (torch tensors) or a raw integer address.
There is no fallback: if libtbpm.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB, LIB_DEBUG

SQUARE, HONEYCOMB, CUBIC = 0, 1, 2
PATH_AUTO, PATH_STENCIL, PATH_CSR = 0, 1, 2
C64, C128 = 0, 1
STATES_RANDOM, STATES_SITES = 0, 1
SEQUENTIAL, CONCURRENT_M, CONCURRENT_S, CONCURRENT_E = 0, 1, 2, 3
DOS_JACKSON, DOS_FOURIER = 0, 1
WINDOW_NONE, WINDOW_HANN = 0, 1
RECON_FP64, RECON_TENSOR = 0, 1

STATUS = {0: "TBPM_OK", -1: "TBPM_EINVAL", -2: "TBPM_ENOMEM", -3: "TBPM_ECUDA", -4: "TBPM_ETIMEOUT",
          -5: "TBPM_EUNSUPPORTED", -6: "TBPM_EBUSY", -7: "TBPM_ECANCELLED"}


class TbpmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class LatticeDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("path", C.c_int32), ("L", C.c_int64 * 3), ("pbc", C.c_int32 * 3),
                ("reserved", C.c_int32), ("t", C.c_double), ("W", C.c_double),
                ("vacancy_frac", C.c_double), ("seed", C.c_uint64), ("cutoff", C.c_double),
                ("decay", C.c_double)]


class LatticeProps(C.Structure):
    _fields_ = [("n_full", C.c_int64), ("n_sites", C.c_int64), ("n_bonds", C.c_int64),
                ("path", C.c_int32), ("coordination", C.c_int32), ("E_min", C.c_double),
                ("E_max", C.c_double), ("H0", C.c_double), ("half_width", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int32), ("max_queue", C.c_int32),
                ("recon", C.c_int32), ("reserved", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("precision", C.c_int32), ("states", C.c_int32), ("n_states", C.c_int32),
                ("form", C.c_int32), ("state_seed", C.c_uint64), ("sites", C.POINTER(C.c_int64)),
                ("n_moments", C.c_int64), ("n_steps", C.c_int64), ("tau", C.c_double),
                ("time_block", C.c_int32), ("dos_method", C.c_int32), ("window", C.c_int32),
                ("recon", C.c_int32)]


_lib = None
_P = C.c_void_p


def load():
    """Load libtbpm.so (built in-tree by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"{LIB} is missing: build it with __graft_entry__.build() "
                          "(there is no fallback implementation)")
    _lib = _bind(C.CDLL(LIB))
    return _lib


_lib_debug = None


def load_debug():
    """Load the index-checked libtbpm_debug.so (paper_2510_17432_gb300._build.build(debug=True))."""
    global _lib_debug
    if _lib_debug is None:
        if not os.path.exists(LIB_DEBUG):
            raise ImportError(f"{LIB_DEBUG} is missing: build it with _build.build(debug=True)")
        _lib_debug = _bind(C.CDLL(LIB_DEBUG))
    return _lib_debug


def _bind(lib):
    sig = {
        "tbpm_create": (C.c_int, [C.POINTER(_P), C.c_int]),
        "tbpm_destroy": (C.c_int, [_P]),
        "tbpm_last_error": (C.c_char_p, []),
        "tbpm_stream": (_P, [_P]),
        "tbpm_sync": (C.c_int, [_P]),
        "tbpm_launch_count": (C.c_int64, [_P]),
        "tbpm_profile": (C.c_int, [_P, C.c_int]),
        "tbpm_set_fusion": (C.c_int, [_P, C.c_int]),
        "tbpm_profile_read": (C.c_int, [_P, C.POINTER(C.c_double)]),
        "tbpm_lattice_create": (C.c_int, [_P, C.POINTER(LatticeDesc), C.POINTER(_P)]),
        "tbpm_lattice_destroy": (C.c_int, [_P]),
        "tbpm_lattice_info": (C.c_int, [_P, C.POINTER(LatticeProps)]),
        "tbpm_lattice_export": (C.c_int, [_P, _P, _P, _P]),
        "tbpm_lattice_taps": (C.c_int, [_P, _P, _P]),
        "tbpm_moment_pass_kind": (C.c_int, [_P, _P, C.POINTER(Request), C.POINTER(C.c_int)]),
        "tbpm_fp32_fma_peak": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "tbpm_debug_status": (C.c_int, [_P, C.POINTER(C.c_uint64)]),
        "tbpm_wait_probe": (C.c_int, [_P, C.c_int, C.c_double]),
        "tbpm_states_export": (C.c_int, [_P, _P, C.POINTER(Request), _P, _P]),
        "tbpm_apply_hopping": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P]),
        "tbpm_moments": (C.c_int, [_P, _P, C.POINTER(Request), _P]),
        "tbpm_moments_device": (C.c_int, [_P, _P, C.POINTER(Request), _P]),
        "tbpm_correlation": (C.c_int, [_P, _P, C.POINTER(Request), _P]),
        "tbpm_correlation_device": (C.c_int, [_P, _P, C.POINTER(Request), _P]),
        "tbpm_dos": (C.c_int, [_P, _P, C.POINTER(Request), _P, C.c_int64, _P]),
        "tbpm_dos_device": (C.c_int, [_P, _P, C.POINTER(Request), _P, C.c_int64, _P]),
        "tbpm_moment_step_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_double,
                                                C.c_double, _P, C.c_int, C.c_int, _P, _P, _P, C.c_int64,
                                                C.c_int64, _P]),
        "tbpm_server_create": (C.c_int, [_P, C.POINTER(ServerConfig), C.POINTER(_P)]),
        "tbpm_server_destroy": (C.c_int, [_P]),
        "tbpm_submit": (C.c_int, [_P, C.POINTER(LatticeDesc), C.POINTER(Request), _P, C.c_int64,
                                  C.POINTER(C.c_uint64)]),
        "tbpm_wait": (C.c_int, [_P, C.c_uint64, C.c_int64, _P, C.c_size_t, C.POINTER(C.c_double)]),
        "tbpm_server_stats": (C.c_int, [_P, C.POINTER(C.c_int64)]),
        "tbpm_quasi_eigenstates": (C.c_int, [_P, _P, C.POINTER(Request), _P, C.c_int64, _P]),
        "tbpm_conductivity": (C.c_int, [_P, _P, C.POINTER(Request), C.c_int, _P, C.c_int64, _P, _P]),
        "tbpm_conductivity_overlap": (C.c_int, [_P, _P, C.POINTER(Request), C.c_int, _P, C.c_int64, _P, _P, _P]),
        "tbpm_fermi_apply": (C.c_int, [_P, _P, C.POINTER(Request), C.c_double, C.c_double, C.c_int, _P]),
        "tbpm_optical_conductivity": (C.c_int, [_P, _P, C.POINTER(Request), C.c_int, C.c_int, C.c_double,
                                                C.c_double, C.c_double, C.c_int64, _P, _P]),
        "tbpm_polarization": (C.c_int, [_P, _P, C.POINTER(Request), _P, C.c_double, C.c_double, _P, C.c_int64,
                                        _P, _P]),
        "tbpm_charge_density": (C.c_int, [_P, _P, C.POINTER(Request), C.c_double, C.c_double, _P]),
        "tbpm_set_pass_states": (C.c_int, [_P, C.c_int]),
        "tbpm_fusion_report": (C.c_int, [_P, C.POINTER(C.c_double)]),
        "tbpm_set_graphs": (C.c_int, [_P, C.c_int]),
        "tbpm_set_block_buffering": (C.c_int, [_P, C.c_int]),
        "tbpm_truncation_order": (C.c_int64, [C.c_double]),
        "tbpm_block_counts": (C.c_int, [C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_int64)]),
        "tbpm_block_opt": (C.c_int64, [C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int64]),
        "tbpm_block_autotune": (C.c_int, [_P, _P, C.POINTER(Request), C.c_int64, C.POINTER(C.c_int64),
                                          C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def exported_symbols():
    """Names of every entry point this binding wraps (all declared in include/tbpm.h)."""
    return ["tbpm_create", "tbpm_destroy", "tbpm_last_error", "tbpm_stream", "tbpm_sync",
            "tbpm_launch_count", "tbpm_set_fusion", "tbpm_profile", "tbpm_profile_read", "tbpm_lattice_create", "tbpm_lattice_destroy", "tbpm_lattice_info",
            "tbpm_lattice_export", "tbpm_lattice_taps", "tbpm_moment_pass_kind", "tbpm_fp32_fma_peak", "tbpm_debug_status", "tbpm_wait_probe", "tbpm_states_export", "tbpm_apply_hopping", "tbpm_moments",
            "tbpm_moments_device", "tbpm_correlation", "tbpm_correlation_device", "tbpm_dos",
            "tbpm_dos_device", "tbpm_quasi_eigenstates", "tbpm_conductivity", "tbpm_conductivity_overlap",
            "tbpm_fermi_apply",
            "tbpm_optical_conductivity", "tbpm_polarization", "tbpm_charge_density", "tbpm_set_pass_states", "tbpm_fusion_report", "tbpm_set_graphs", "tbpm_set_block_buffering", "tbpm_moment_step_noalloc", "tbpm_truncation_order", "tbpm_block_counts", "tbpm_block_opt",
            "tbpm_block_autotune", "tbpm_server_create", "tbpm_server_destroy", "tbpm_submit", "tbpm_wait",
            "tbpm_server_stats"]


def _check(status: int, lib=None):
    if status != 0:
        raise TbpmError(status, (lib or load()).tbpm_last_error().decode(errors="replace"))


def _host_ptr(a: np.ndarray | None):
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return a.ctypes.data_as(C.c_void_p)


def _out_ptr(a: np.ndarray | None, needed: int, what: str):
    """Host pointer of an output buffer that the library fills with `needed` bytes; a buffer
    too small for them is refused here, before the library could write past its end."""
    if a is not None and a.nbytes < needed:
        raise ValueError(f"{what}: the buffer holds {a.nbytes} bytes, the request writes {needed}")
    return _host_ptr(a)


def _dev_ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- context
def tbpm_create(device: int = 0):
    h = _P()
    _check(load().tbpm_create(C.byref(h), int(device)))
    return h


def tbpm_destroy(ctx):
    _check(load().tbpm_destroy(ctx))


def tbpm_last_error() -> str:
    return load().tbpm_last_error().decode(errors="replace")


def tbpm_stream(ctx) -> int:
    return load().tbpm_stream(ctx) or 0


def tbpm_sync(ctx):
    _check(load().tbpm_sync(ctx))


def tbpm_launch_count(ctx) -> int:
    return int(load().tbpm_launch_count(ctx))


def tbpm_set_fusion(ctx, mode: int):
    """0 = one step per pass, 1..3 = fused variants (see include/tbpm.h)."""
    _check(load().tbpm_set_fusion(ctx, int(mode)))


def tbpm_profile(ctx, enable: bool):
    _check(load().tbpm_profile(ctx, int(bool(enable))))


def tbpm_profile_read(ctx) -> dict:
    out = (C.c_double * 6)()
    _check(load().tbpm_profile_read(ctx, out))
    return {"recurrence_ms": out[0], "recurrence_launches": int(out[1]),
            "recon_ms": out[2], "recon_launches": int(out[3]),
            "fused_ms": out[4], "fused_launches": int(out[5])}


# ---------------------------------------------------------------- lattice
def lattice_desc(kind, L, t=1.0, W=0.0, vacancy_frac=0.0, seed=0, pbc=(1, 1, 1), path=PATH_AUTO,
                 cutoff=0.0, decay=0.0) -> LatticeDesc:
    L = tuple(int(v) for v in L) + (1,) * (3 - len(L))
    pbc = tuple(int(bool(v)) for v in pbc) + (1,) * (3 - len(pbc))
    return LatticeDesc(int(kind), int(path), (C.c_int64 * 3)(*L), (C.c_int32 * 3)(*pbc), 0,
                       float(t), float(W), float(vacancy_frac), int(seed) & 0xFFFFFFFFFFFFFFFF,
                       float(cutoff), float(decay))


def tbpm_lattice_create(ctx, desc: LatticeDesc):
    h = _P()
    _check(load().tbpm_lattice_create(ctx, C.byref(desc), C.byref(h)))
    return h


def tbpm_lattice_destroy(lat):
    _check(load().tbpm_lattice_destroy(lat))


def tbpm_lattice_info(lat) -> LatticeProps:
    p = LatticeProps()
    _check(load().tbpm_lattice_info(lat, C.byref(p)))
    return p


def tbpm_lattice_export(lat, compact=None, V=None, nbr=None):
    _check(load().tbpm_lattice_export(lat, _host_ptr(compact), _host_ptr(V), _host_ptr(nbr)))


def tbpm_lattice_taps(lat):
    """(offsets [z][4] int32, t [z] float64) of the lattice's neighbour slots."""
    z = tbpm_lattice_info(lat).coordination
    off = np.zeros((z, 4), np.int32)
    t = np.zeros(z, np.float64)
    _check(load().tbpm_lattice_taps(lat, _host_ptr(off), _host_ptr(t)))
    return off, t


# ---------------------------------------------------------------- requests
def request(n_states=1, precision=C64, form=CONCURRENT_M, n_moments=0, n_steps=0, state_seed=1,
            sites=None, tau=0.0, time_block=0, dos_method=DOS_JACKSON, window=WINDOW_NONE,
            recon=RECON_FP64):
    """Build a Request; keeps a reference to the site array so the pointer stays valid."""
    r = Request()
    r.precision = precision
    r.form = form
    r.state_seed = int(state_seed) & 0xFFFFFFFFFFFFFFFF
    r.n_moments = int(n_moments)
    r.n_steps = int(n_steps)
    r.tau = float(tau)
    r.time_block = int(time_block)
    r.dos_method = dos_method
    r.window = window
    r.recon = recon
    if sites is not None:
        arr = np.ascontiguousarray(sites, dtype=np.int64)
        r.states = STATES_SITES
        r.n_states = arr.size
        r.sites = arr.ctypes.data_as(C.POINTER(C.c_int64))
        r._sites_keepalive = arr
    else:
        r.states = STATES_RANDOM
        r.n_states = int(n_states)
        r.sites = None
    return r


def tbpm_states_export(ctx, lat, req: Request, out=None, draws=None):
    _check(load().tbpm_states_export(ctx, lat, C.byref(req), _host_ptr(out), _host_ptr(draws)))


def tbpm_apply_hopping(ctx, lat, precision: int, n_states: int, x: np.ndarray, y: np.ndarray):
    _check(load().tbpm_apply_hopping(ctx, lat, int(precision), int(n_states), _host_ptr(x), _host_ptr(y)))


def tbpm_moments(ctx, lat, req: Request, mu: np.ndarray):
    """mu: [S][M][2] float64 (re, im)."""
    S, M = int(req.n_states), int(req.n_moments)
    need = 16 * S * M if 1 <= S <= 32 and M >= 2 and M % 2 == 0 else 0  # else the library refuses
    _check(load().tbpm_moments(ctx, lat, C.byref(req), _out_ptr(mu, need, "tbpm_moments")))


def tbpm_moments_device(ctx, lat, req: Request, d_mu):
    _check(load().tbpm_moments_device(ctx, lat, C.byref(req), _dev_ptr(d_mu)))


def tbpm_correlation(ctx, lat, req: Request, Cout: np.ndarray):
    """Cout: [S][N_t+1][2] float64 (or [S][N_t+1] complex128)."""
    S, Nt = int(req.n_states), int(req.n_steps)
    need = 16 * S * (Nt + 1) if 1 <= S <= 32 and Nt >= 1 else 0
    _check(load().tbpm_correlation(ctx, lat, C.byref(req), _out_ptr(Cout, need, "tbpm_correlation")))


def tbpm_correlation_device(ctx, lat, req: Request, d_C):
    _check(load().tbpm_correlation_device(ctx, lat, C.byref(req), _dev_ptr(d_C)))


def tbpm_dos(ctx, lat, req: Request, energies: np.ndarray, D: np.ndarray):
    """energies: [n_energies] float64 (converted if needed); D: [S][n_energies] float64."""
    e = np.ascontiguousarray(energies, dtype=np.float64)  # no copy for a float64 C-ordered array
    S = int(req.n_states)
    need = 8 * S * e.size if 1 <= S <= 32 else 0
    _check(load().tbpm_dos(ctx, lat, C.byref(req), _host_ptr(e), int(e.size), _out_ptr(D, need, "tbpm_dos")))


def tbpm_dos_device(ctx, lat, req: Request, d_energies, n_energies: int, d_D):
    _check(load().tbpm_dos_device(ctx, lat, C.byref(req), _dev_ptr(d_energies), int(n_energies), _dev_ptr(d_D)))


def tbpm_quasi_eigenstates(ctx, lat, req: Request, energies: np.ndarray, out: np.ndarray):
    """out: [n_energies][S][n_sites] complex64 (C64) or complex128 (C128)."""
    e = np.ascontiguousarray(energies, dtype=np.float64)
    _check(load().tbpm_quasi_eigenstates(ctx, lat, C.byref(req), _host_ptr(e), int(e.size), _host_ptr(out)))


def tbpm_conductivity(ctx, lat, req: Request, direction: int, energies: np.ndarray, C_out: np.ndarray | None,
                      sigma: np.ndarray):
    """C_out: [S][n_energies][n_steps+1] complex128 or None; sigma: [S][n_energies] float64."""
    e = np.ascontiguousarray(energies, dtype=np.float64)
    _check(load().tbpm_conductivity(ctx, lat, C.byref(req), int(direction), _host_ptr(e), int(e.size),
                                    _host_ptr(C_out), _host_ptr(sigma)))


PASS_STENCIL, PASS_ELL, PASS_TAPS, PASS_SWEEP, PASS_ROWS, PASS_TILES = 0, 1, 2, 3, 4, 5
DEBUG_KERNELS = {1: "stencil units", 2: "ELL neighbour index", 3: "sweep store", 4: "sweep row copy",
                 5: "serving units"}


def tbpm_debug_status(ctx, lib=None) -> list:
    """The debug build's three index-check words (recurrence passes, register sweep, serving),
    read and cleared; raises TbpmError(TBPM_EUNSUPPORTED) on the regular library."""
    words = (C.c_uint64 * 3)()
    _check((lib or load()).tbpm_debug_status(ctx, words), lib)
    return [int(w) for w in words]


def tbpm_wait_probe(ctx, arrive: bool, budget_s: float):
    """One-warp run of the register sweep's bounded mbarrier wait; raises
    TbpmError(TBPM_ETIMEOUT) when nothing arrives within budget_s seconds."""
    _check(load().tbpm_wait_probe(ctx, int(bool(arrive)), float(budget_s)))


def decode_debug_word(word: int):
    """(kernel name, index) of a failed check, or None for a clean word."""
    if word == 0:
        return None
    return DEBUG_KERNELS.get(word >> 48, f"kernel {word >> 48}"), word & 0xFFFFFFFFFFFF


def tbpm_moment_pass_kind(ctx, lat, req: Request) -> int:
    """The kernel family that carries the request's moment recurrence (PASS_* constants)."""
    k = C.c_int(0)
    _check(load().tbpm_moment_pass_kind(ctx, lat, C.byref(req), C.byref(k)))
    return k.value


def tbpm_fp32_fma_peak(ctx) -> tuple:
    """Measured FP32 FMA throughput (scalar, packed f32x2) of the context's device in TFLOP/s."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _check(load().tbpm_fp32_fma_peak(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def tbpm_conductivity_overlap(ctx, lat, req: Request, direction: int, energies: np.ndarray,
                              C_out: np.ndarray | None, sigma: np.ndarray, overlap: np.ndarray | None):
    """As tbpm_conductivity; overlap: [S][n_energies] complex128 (<psi|Psi(E)> as the device used it) or None."""
    e = np.ascontiguousarray(energies, dtype=np.float64)
    _check(load().tbpm_conductivity_overlap(ctx, lat, C.byref(req), int(direction), _host_ptr(e), int(e.size),
                                            _host_ptr(C_out), _host_ptr(sigma), _host_ptr(overlap)))


def tbpm_fermi_apply(ctx, lat, req: Request, mu: float, kT: float, sqrt_f: bool, out: np.ndarray):
    """out: [S][n_sites] complex64 (C64) or complex128 (C128)."""
    _check(load().tbpm_fermi_apply(ctx, lat, C.byref(req), float(mu), float(kT), int(bool(sqrt_f)), _host_ptr(out)))


def tbpm_optical_conductivity(ctx, lat, req: Request, alpha: int, beta: int, mu: float, kT: float,
                              omega_max: float, n_omega: int, C_out: np.ndarray | None, sigma: np.ndarray):
    """C_out: [S][n_steps+1] complex128 or None; sigma: [S][n_omega] complex128 (Re + i Im)."""
    _check(load().tbpm_optical_conductivity(ctx, lat, C.byref(req), int(alpha), int(beta), float(mu), float(kT),
                                            float(omega_max), int(n_omega), _host_ptr(C_out), _host_ptr(sigma)))


def tbpm_polarization(ctx, lat, req: Request, q, mu: float, kT: float, omegas: np.ndarray,
                      C_out: np.ndarray | None, Pi: np.ndarray):
    """q: 3 floats; C_out: [S][n_steps+1] complex128 or None; Pi: [S][n_omega] complex128."""
    qa = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(3))
    w = np.ascontiguousarray(omegas, dtype=np.float64)
    _check(load().tbpm_polarization(ctx, lat, C.byref(req), _host_ptr(qa), float(mu), float(kT), _host_ptr(w),
                                    int(w.size), _host_ptr(C_out), _host_ptr(Pi)))


def tbpm_set_graphs(ctx, enable: bool):
    _check(load().tbpm_set_graphs(ctx, int(bool(enable))))


def tbpm_set_block_buffering(ctx, enable: bool):
    _check(load().tbpm_set_block_buffering(ctx, int(bool(enable))))


def tbpm_fusion_report(ctx) -> dict:
    """ms per step of each fusion mode timed by the last autotune (mode -> ms)."""
    out = (C.c_double * 16)()
    _check(load().tbpm_fusion_report(ctx, out))
    return {m: out[m] for m in range(16) if out[m] >= 0.0}


def tbpm_set_pass_states(ctx, max_states: int):
    _check(load().tbpm_set_pass_states(ctx, int(max_states)))


def tbpm_charge_density(ctx, lat, req: Request, mu: float, kT: float, rho: np.ndarray):
    """rho: [S][n_sites] float64."""
    _check(load().tbpm_charge_density(ctx, lat, C.byref(req), float(mu), float(kT), _host_ptr(rho)))


def tbpm_moment_step_noalloc(kind, L, pbc, t_scaled, diag_const, d_diag, precision, n_states, d_cur,
                             d_prev_out, d_mu, n_moments, step, stream=0):
    """One allocation-free moment pass; every buffer is the caller's (see include/tbpm.h)."""
    L = tuple(int(v) for v in L) + (1,) * (3 - len(L))
    pbc = tuple(int(bool(v)) for v in pbc) + (1,) * (3 - len(pbc))
    _check(load().tbpm_moment_step_noalloc(int(kind), (C.c_int64 * 3)(*L), (C.c_int32 * 3)(*pbc), float(t_scaled),
                                           float(diag_const), _dev_ptr(d_diag), int(precision), int(n_states),
                                           _dev_ptr(d_cur), _dev_ptr(d_prev_out), _dev_ptr(d_mu), int(n_moments),
                                           int(step), C.c_void_p(int(stream)) if stream else None))


# ---------------------------------------------------------------- serving
def tbpm_server_create(ctx, hbm_budget_bytes=0, max_active=0, max_queue=0, recon=RECON_FP64):
    h = _P()
    cfg = ServerConfig(int(hbm_budget_bytes), int(max_active), int(max_queue), int(recon), 0)
    _check(load().tbpm_server_create(ctx, C.byref(cfg), C.byref(h)))
    return h


def tbpm_server_destroy(srv):
    _check(load().tbpm_server_destroy(srv))


def tbpm_submit(srv, desc: LatticeDesc, req: Request, energies: np.ndarray) -> int:
    t = C.c_uint64()
    e = np.ascontiguousarray(energies, dtype=np.float64)
    _check(load().tbpm_submit(srv, C.byref(desc), C.byref(req), _host_ptr(e), int(e.size), C.byref(t)))
    return int(t.value)


def tbpm_wait(srv, ticket: int, D: np.ndarray, timeout_us: int = -1):
    """Fills D ([S][n_energies]) and returns (queued_us, run_us, total_us)."""
    lat = (C.c_double * 3)()
    _check(load().tbpm_wait(srv, C.c_uint64(ticket), int(timeout_us), _host_ptr(D), int(D.size), lat))
    return float(lat[0]), float(lat[1]), float(lat[2])


def tbpm_server_stats(srv) -> dict:
    out = (C.c_int64 * 7)()
    _check(load().tbpm_server_stats(srv, out))
    return dict(zip(("queued", "active", "completed", "launches", "reserved_bytes", "budget_bytes", "gpu_us"),
                    (int(v) for v in out)))


# ---------------------------------------------------------------- cost model
def tbpm_truncation_order(tau: float) -> int:
    return int(load().tbpm_truncation_order(float(tau)))


def tbpm_block_counts(n_steps: int, b: int, tau: float) -> tuple:
    out = (C.c_int64 * 3)()
    _check(load().tbpm_block_counts(int(n_steps), int(b), float(tau), out))
    return tuple(int(v) for v in out)


def tbpm_block_opt(n_steps: int, tau: float, t_amxsy: float, t_axpy: float, b_max: int) -> int:
    return int(load().tbpm_block_opt(int(n_steps), float(tau), float(t_amxsy), float(t_axpy), int(b_max)))


def tbpm_block_autotune(ctx, lat, req: Request, n_steps: int):
    """Returns (b_opt, t_amxsy_ms, t_axpy_ms) measured on the device."""
    b = C.c_int64()
    t = (C.c_double * 2)()
    _check(load().tbpm_block_autotune(ctx, lat, C.byref(req), int(n_steps), C.byref(b), t))
    return int(b.value), float(t[0]), float(t[1])
