"""NVTX ranges of the library: every public compute call opens a range named after itself, and
the recurrence and reconstruction phases open ranges inside it, so a profiler can attribute
kernels to calls and phases (ncu --nvtx).  A test-only NVTX handler (tests/nvtx_recorder.c, built
here with gcc) records the range calls in a child process started with NVTX_INJECTION64_PATH; the
test checks the names and that every range is closed when its call returns, error returns
included.

Without a GPU: calls rejected for NULL arguments still open and close their range.  With a GPU:
a DOS request opens tbpm_dos with the recurrence and reconstruction phases inside, and all ranges
are closed after each call."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "nvtx_recorder.c")

PRELUDE = """
import ctypes as C, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2510_17432_gb300 import capi
lib = capi.load()
rec = C.CDLL({recorder!r})
rec.nvtx_recorder_log.restype = C.c_char_p
def dump():
    print("__NVTX_LOG__")
    print(rec.nvtx_recorder_log().decode(), end="")
"""


def _cuda_include():
    nvcc = shutil.which("nvcc")
    for home in (os.environ.get("CUDA_HOME"), os.path.dirname(os.path.dirname(nvcc)) if nvcc else None,
                 "/usr/local/cuda"):
        if home and os.path.exists(os.path.join(home, "include", "nvtx3", "nvToolsExt.h")):
            return os.path.join(home, "include")
    pytest.skip("nvtx3 headers not found")


@pytest.fixture(scope="module")
def recorder(tmp_path_factory):
    import __graft_entry__
    __graft_entry__.build()
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    out = str(tmp_path_factory.mktemp("nvtx") / "libnvtx_recorder.so")
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I", _cuda_include(), "-o", out, SRC, "-lpthread"],
                   check=True, capture_output=True)
    return out


def run_child(recorder, body: str) -> list:
    env = dict(os.environ, NVTX_INJECTION64_PATH=recorder)
    code = PRELUDE.format(root=ROOT, recorder=recorder) + body
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return r.stdout.split("__NVTX_LOG__\n", 1)[1].splitlines()


def check_closed(lines: list):
    """Pushes and pops nest and balance; every started range ends exactly once."""
    depth, open_ids = 0, {}
    for ln in lines:
        if ln.startswith("push "):
            depth += 1
        elif ln == "pop":
            depth -= 1
            assert depth >= 0, lines
        elif ln.startswith("start "):
            _, rid, name = ln.split(" ", 2)
            assert rid not in open_ids
            open_ids[rid] = name
        elif ln.startswith("end "):
            rid = ln.split()[1]
            assert rid in open_ids, (ln, lines)
            del open_ids[rid]
    assert depth == 0 and not open_ids, (depth, open_ids)


def test_rejected_calls_open_and_close_their_range(recorder):
    lines = run_child(recorder, """
out = C.c_void_p()
assert lib.tbpm_lattice_create(None, None, C.byref(out)) == -1
assert lib.tbpm_moments(None, None, None, None) == -1
assert lib.tbpm_dos(None, None, None, None, 0, None) == -1
dump()
""")
    assert lines == ["push tbpm_lattice_create", "pop", "push tbpm_moments", "pop", "push tbpm_dos", "pop"]


@pytest.mark.gpu
def test_dos_call_holds_its_phase_ranges(recorder):
    lines = run_child(recorder, """
ctx = capi.tbpm_create(0)
lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (64, 48), t=-2.7, W=0.5, seed=3))
props = capi.tbpm_lattice_info(lat)
E = np.linspace(-8.0, 8.0, 64)
for _ in range(2):
    D = np.zeros((4, 64))
    capi.tbpm_dos(ctx, lat, capi.request(n_states=4, n_moments=256, state_seed=3), E, D)
    assert np.all(np.isfinite(D))
capi.tbpm_lattice_destroy(lat)
capi.tbpm_destroy(ctx)
dump()
""")
    check_closed(lines)
    assert lines[0] == "push tbpm_lattice_create"
    starts = [ln for ln in lines if ln.startswith("push tbpm_dos")]
    assert len(starts) == 2
    # inside each tbpm_dos range: a recurrence phase, then a reconstruction phase
    i = lines.index("push tbpm_dos")
    depth, j = 0, i
    for j in range(i, len(lines)):
        depth += 1 if lines[j].startswith("push ") else -1 if lines[j] == "pop" else 0
        if depth == 0:
            break
    inner = [ln.split(" ", 2)[2] for ln in lines[i:j] if ln.startswith("start ")]
    assert "recurrence" in inner and "reconstruction" in inner
    assert inner.index("recurrence") < inner.index("reconstruction")
