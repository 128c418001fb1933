"""The allocation-free moment step against the regular moments entry point.

tbpm_moment_step_noalloc is for callers that cannot let a library allocate device memory:
applications that keep nearly all HBM in their own arena, loops where a cudaMalloc or
cudaFree could synchronise the device, and plugin hosts that only pass buffers in.  This
test plays such a caller: it owns every buffer (allocated here with torch), drives all M/2
recurrence passes through the C ABI, does so twice in a row (the second run reuses the
library's fixed scratch array after the first), and compares both runs with tbpm_moments on
the same initial states, within the tolerances of the other parity tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-11}


@pytest.mark.parametrize("kind,L,W,prec,S", [(1, (40, 24), 0.0, 0, 8), (0, (33, 20), 1.0, 1, 2),
                                             (2, (6, 5, 7), 2.0, 0, 1), (1, (300, 9), 1.0, 0, 32)])
def test_noalloc_step_matches_moments(kind, L, W, prec, S):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_17432_gb300 import capi

    ctx = capi.tbpm_create(0)
    t = -1.3
    lat = capi.tbpm_lattice_create(ctx, capi.lattice_desc(kind, L, t=t, W=W, seed=11))
    info = capi.tbpm_lattice_info(lat)
    M = 256
    req = capi.request(n_states=S, precision=prec, n_moments=M, state_seed=5)
    ref = np.zeros((S, M, 2))
    capi.tbpm_moments(ctx, lat, req, ref)

    # the same initial states, laid out [site][state] in the caller's own device buffer
    dt = np.complex64 if prec == capi.C64 else np.complex128
    states = np.zeros((S, info.n_sites), dt)
    capi.tbpm_states_export(ctx, lat, req, states)
    x0 = np.ascontiguousarray(states.T)
    diag = None
    if W != 0.0:
        V = np.zeros(info.n_sites)
        capi.tbpm_lattice_export(lat, None, V, None)
        d = (V - info.H0) / info.half_width
        diag = torch.tensor(d.astype(np.float32 if prec == capi.C64 else np.float64), device="cuda")
    capi.tbpm_lattice_destroy(lat)
    capi.tbpm_destroy(ctx)

    dev = torch.device("cuda", 0)
    for run in range(2):
        bufs = [torch.from_numpy(x0).to(dev), torch.empty(x0.shape, dtype=torch.from_numpy(x0).dtype, device=dev)]
        mu = torch.zeros((S, M, 2), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev).cuda_stream
        torch.cuda.synchronize()
        for n in range(M // 2):
            capi.tbpm_moment_step_noalloc(kind, L, (1, 1, 1), t / info.half_width, -info.H0 / info.half_width,
                                          diag, prec, S, bufs[n & 1], bufs[(n + 1) & 1], mu, M, n, stream)
        torch.cuda.synchronize()
        got = mu.cpu().numpy()
        err = np.max(np.abs(got - ref)) / abs(ref[0, 0, 0])
        assert err <= TOL[prec], (run, err)


def test_noalloc_rejects_bad_sizes():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_17432_gb300 import capi
    buf = torch.zeros(64, dtype=torch.complex64, device="cuda")
    mu = torch.zeros(16, dtype=torch.float64, device="cuda")
    for S, M, step in ((3, 8, 0), (64, 8, 0), (1, 7, 0), (1, 8, 4)):
        with pytest.raises(capi.TbpmError):
            capi.tbpm_moment_step_noalloc(0, (8, 8), (1, 1), 0.25, 0.0, None, capi.C64, S, buf, buf, mu, M, step, 0)
