"""Host-side checks of the C ABI (no GPU): the library loads, exports every symbol the
header declares, its structs match the header layout, and its host-only cost-model
entry points agree with the oracle (Sec. II.A truncation, Tab. I counts, b_opt)."""
import ctypes
import math
import os
import re
import subprocess

import pytest

from oracle import bessel, cost

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tbpm.h")


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_17432_gb300 import capi as c
    return c


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(tbpm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("tbpm_create", "tbpm_lattice_create", "tbpm_moments", "tbpm_correlation", "tbpm_dos"):
        assert must in names


def test_library_exports_every_declared_symbol(capi):
    lib = capi.load()
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tbpm_[a-z_0-9]+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(capi.exported_symbols()) <= set(declared_functions())


def test_struct_layout_matches_header(capi):
    # offsets follow the C declarations with natural alignment
    assert ctypes.sizeof(capi.LatticeDesc) == 96
    assert capi.LatticeDesc.t.offset == 48 and capi.LatticeDesc.seed.offset == 72
    assert capi.LatticeDesc.cutoff.offset == 80 and capi.LatticeDesc.decay.offset == 88
    assert ctypes.sizeof(capi.Request) == 72
    assert capi.Request.state_seed.offset == 16 and capi.Request.tau.offset == 48
    assert ctypes.sizeof(capi.LatticeProps) == 64


@pytest.mark.parametrize("tau", [0.5, math.pi, 4 * math.pi, 100.0, 1254 * math.pi, 2048 * math.pi])
def test_truncation_order_matches_oracle(capi, tau):
    assert capi.tbpm_truncation_order(tau) == bessel.truncation_order(tau)


@pytest.mark.parametrize("nt,b", [(30, 1), (30, 5), (30, 7), (100, 40), (1024, 32)])
def test_block_counts_match_table_one(capi, nt, b):
    want = cost.block_counts(nt, b)
    assert capi.tbpm_block_counts(nt, b, math.pi) == (want["amxsy"], want["axpy"], want["dot"])


def test_block_opt_matches_oracle(capi):
    for ta, tx in ((1.0, 0.2), (3.0, 2.0), (1.0, 1.0)):
        assert capi.tbpm_block_opt(512, math.pi, ta, tx, 128) == cost.b_opt(512, ta, tx, b_max=128)


def test_invalid_arguments_fail_cleanly(capi):
    with pytest.raises(capi.TbpmError):
        capi.tbpm_block_counts(0, 1, math.pi)


def test_plain_c_caller(capi, tmp_path):
    """The header is strict C99 (pedantic, warnings as errors) and a C program linked against
    libtbpm.so gets the oracle's truncation orders, Tab. I counts and b_opt, and status codes
    (never a crash) for invalid arguments, all without a GPU."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.join(root, "paper_2510_17432_gb300")
    exe = str(tmp_path / "c_abi_check")
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(root, "include"), "-o", exe, os.path.join(root, "tests", "c_abi_check.c"),
                    "-L", libdir, "-ltbpm", f"-Wl,-rpath,{libdir}", "-lm"], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    out = {ln.split()[0]: ln.split()[1:] for ln in r.stdout.splitlines()}
    assert [int(v) for v in out["truncation"]] == [bessel.truncation_order(k * math.pi) for k in (1, 4, 100)]
    want = cost.block_counts(2048, 40, math.pi)
    assert [int(v) for v in out["counts"]] == [want["amxsy"], want["axpy"], want["dot"]]
    assert int(out["bopt"][0]) == cost.b_opt(2048, 1.0, 0.05, b_max=256)
    assert out["errors"] == ["ok"]


def test_binding_refuses_output_buffers_too_small(capi):
    """The binding checks that a host output buffer holds what the request writes before it
    passes the pointer on; a buffer of the right size reaches the library (here it answers
    TBPM_EINVAL for the NULL context, with no GPU involved)."""
    import numpy as np
    req = capi.request(n_states=4, n_moments=64)
    with pytest.raises(ValueError, match="tbpm_moments"):
        capi.tbpm_moments(None, None, req, np.zeros((4, 64)))          # [S][M] instead of [S][M][2]
    with pytest.raises(capi.TbpmError):
        capi.tbpm_moments(None, None, req, np.zeros((4, 64, 2)))
    creq = capi.request(n_states=2, n_steps=10)
    with pytest.raises(ValueError, match="tbpm_correlation"):
        capi.tbpm_correlation(None, None, creq, np.zeros((2, 10, 2)))   # N_t entries instead of N_t + 1
    with pytest.raises(capi.TbpmError):
        capi.tbpm_correlation(None, None, creq, np.zeros((2, 11), np.complex128))
    E = np.linspace(-1.0, 1.0, 16)
    with pytest.raises(ValueError, match="tbpm_dos"):
        capi.tbpm_dos(None, None, req, E, np.zeros(16))                 # one state's worth for four
    with pytest.raises(capi.TbpmError):
        capi.tbpm_dos(None, None, req, E.astype(np.float32), np.zeros((4, 16)))
    # invalid requests are left to the library, which refuses them before writing anything
    with pytest.raises(capi.TbpmError):
        capi.tbpm_moments(None, None, capi.request(n_states=33, n_moments=8), np.zeros((1, 8, 2)))
