"""Failure detection on the device without a GPU fault.

The kernels fed by TMA copies wait on mbarriers for a bounded time; when a wait expires the
kernel records a code in a status word and returns, the host reports TBPM_ETIMEOUT, and the
context stays usable.  tbpm_wait_probe runs the register sweep's bounded wait in a one-warp
kernel on a barrier that completes (arrive) or that nothing ever arrives at (no copy in flight),
so the expiry path runs for real on the GPU with a short budget, never through a trap or a hang.

Without a GPU: the budget and the context are checked before any device work.  With a GPU: a
completed wait reports OK; an expired one reports TBPM_ETIMEOUT after about its budget; the report
clears the status word; and a moment request on the register sweep run after the expiry equals,
bit for bit, the same request run before it."""
import ctypes as C
import time

import numpy as np
import pytest


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_17432_gb300 import capi as c
    return c


def test_probe_arguments_are_checked_before_device_work(capi):
    lib = capi.load()
    assert lib.tbpm_wait_probe(None, 0, 0.01) == -1
    # a non-NULL dummy handle is never dereferenced when the budget is rejected
    for budget in (0.0, -1.0, 2.5, float("nan")):
        assert lib.tbpm_wait_probe(C.c_void_p(1), 0, budget) == -1, budget


@pytest.mark.gpu
def test_expired_wait_is_reported_and_the_context_stays_usable(capi):
    ctx = capi.tbpm_create(0)
    try:
        capi.tbpm_set_fusion(ctx, 8)
        lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(1, (100, 64), t=-2.7, W=1.0, seed=3))
        req = capi.request(n_states=8, n_moments=256, state_seed=5)
        assert capi.tbpm_moment_pass_kind(ctx, lat, req) == capi.PASS_SWEEP
        before = np.zeros((8, 256, 2))
        capi.tbpm_moments(ctx, lat, req, before)

        capi.tbpm_wait_probe(ctx, True, 0.5)  # the barrier completes: no error

        budget = 0.05
        t0 = time.perf_counter()
        with pytest.raises(capi.TbpmError) as ei:
            capi.tbpm_wait_probe(ctx, False, budget)
        dt = time.perf_counter() - t0
        assert ei.value.status == -4, str(ei.value)
        assert "bounded wait" in str(ei.value)
        assert 0.8 * budget <= dt < 5.0, dt

        capi.tbpm_wait_probe(ctx, True, 0.5)  # the report cleared the status word
        after = np.zeros_like(before)
        capi.tbpm_moments(ctx, lat, req, after)
        assert np.array_equal(before, after)
        assert np.all(np.isfinite(after)) and abs(after[0, 0, 0] - 1.0) < 1e-5
        capi.tbpm_lattice_destroy(lat)
    finally:
        capi.tbpm_destroy(ctx)
