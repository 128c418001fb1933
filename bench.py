#!/usr/bin/env python
"""Benchmark of the concurrent Chebyshev propagation hot path on GB300.

Default workload: graphene honeycomb 2048 x 2048 cells (8,388,608 sites), t = -2.7 eV, clean,
8 random-phase complex64 states with FP64 moment reductions, 4096 Chebyshev moments by the
moment-based concurrent form with the cost-halving identity (2048 matrix applications), and the
Jackson DOS on 8192 energies.  One step = lattice build + states + recurrence with fused moments
+ reconstruction, through the C ABI.

Metric: site-updates/s, one site-update = one Chebyshev recurrence step applied to one site of one
state.  Printed as one JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

WORKLOADS = {
    "graphene2048": wl.GRAPHENE_2048,
    "graphene1024": wl.Workload("honeycomb1024x1024_S8_M256", wl.honeycomb(1024, 1024, t=-2.7), n_states=8,
                                n_moments=256, precision=wl.C64, n_steps=70, n_energies=1024),
    "recon_probe": wl.Workload("honeycomb256x256_S8_M4096_E8192", wl.honeycomb(256, 256, t=-2.7), n_states=8,
                               n_moments=4096, precision=wl.C64, n_steps=0, n_energies=8192),
    "graphene512": wl.Workload("honeycomb512x512_S8_M1024", wl.honeycomb(512, 512, t=-2.7), n_states=8,
                               n_moments=1024, precision=wl.C64, n_steps=300, n_energies=2048),
    "graphene22528": wl.GRAPHENE_22528,
    # the 1.015e9-site workload's state count and disorder on a 2048 x 2048 lattice (profiling case)
    "graphene2048_W1_S4": wl.Workload("honeycomb2048x2048_W1_S4_M256", wl.honeycomb(2048, 2048, t=-2.7, W=1.0),
                                      n_states=4, n_moments=256, precision=wl.C64, n_steps=0, n_energies=1024),
    "square64": wl.SQUARE_64,
    "vacancy4096": wl.GRAPHENE_4096_VAC,
    "dense61": wl.dense_honeycomb(61),
    "dense124": wl.dense_honeycomb(124),
    "dense235": wl.dense_honeycomb(235),
    "dense235_small": wl.dense_honeycomb(235, n_steps=64, L=(1024, 2048)),   # profiling case
    "vacancy2048": wl.Workload("honeycomb2048x2048_vac1pct_W2_Nt512", wl.honeycomb(2048, 2048, t=-2.7, W=2.0,
                                                                                 vacancy_frac=0.01, path=wl.PATH_CSR),
                               n_states=1, n_moments=0, precision=wl.C64, n_steps=512, n_energies=16),
    "vacancy1024": wl.Workload("honeycomb1024x1024_vac1pct_W2_Nt256", wl.honeycomb(1024, 1024, t=-2.7, W=2.0,
                                                                                 vacancy_frac=0.01, path=wl.PATH_CSR),
                               n_states=1, n_moments=0, precision=wl.C64, n_steps=256, n_energies=16),
}
# source files that define each measured kernel family (their hash keys the stored ncu traffic)
KERNEL_SRCS = {
    "k_moment_stencil": ("cheb.cu", "stencil.cuh"),
    "k_fused_cols": ("fused.cu",),
    "k_fused_rows": ("fused.cu",),
    "k_sweep": ("sweep.cu",),
}
# Chebyshev steps per launch and kernel of each fusion mode of the moment pass
FUSION_STEPS = {1: 4, 2: 2, 3: 2, 4: 2, 5: 4, 6: 4, 7: 2, 8: 4, 9: 4, 10: 4}
FUSION_KERNELS = {1: "k_fused_cols (4 Chebyshev steps per pass, 2-D tiles)",
                  2: "k_fused_cols (2 Chebyshev steps per pass, 2-D tiles)",
                  3: "k_fused_rows<128> (2 Chebyshev steps per pass, row sweep)",
                  4: "k_fused_rows<256> (2 Chebyshev steps per pass, row sweep)",
                  5: "k_fused_rowsK<128, 4> (4 Chebyshev steps per pass, row sweep)",
                  6: "k_fused_rowsK<256, 4> (4 Chebyshev steps per pass, row sweep)",
                  7: "k_fused_rowsK<256, 2> (2 Chebyshev steps per pass, row sweep)",
                  8: "k_sweep_moments<128, 4> (4 Chebyshev steps per pass, register sweep, TMA rows)",
                  9: "k_sweep_moments<192, 4> (4 Chebyshev steps per pass, register sweep, TMA rows)",
                  10: "k_sweep_moments<256, 4> (4 Chebyshev steps per pass, register sweep, TMA rows)"}
FUSION_TRAFFIC_FAMILY = {8: "k_sweep", 9: "k_sweep", 10: "k_sweep"}
TRAFFIC = os.path.join(ROOT, "profiles", "roofline_traffic.json")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tbpm", choices=["tbpm", "reference"])
    p.add_argument("--workload", default="graphene2048", choices=sorted(WORKLOADS))
    p.add_argument("--recon", default="tensor", choices=["fp64", "tensor"])
    p.add_argument("--no-sequential", action="store_true", help="skip the sequential-form comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--fusion", type=int, default=8,
                   help="moment-pass fusion mode: 0 = one step per pass, 1 = 4-step tiles, 2 = 2-step tiles, "
                        "3/4 = 2-step row sweep, 5/6 = 4-step row sweep, 7 = 2-step sweep (K-step code), "
                        "8/9/10 = 4-step register sweep (128/192/256 threads), -1 = autotuned")
    p.add_argument("--serving", action="store_true", help="serving stream: Poisson arrivals, p50/p99 latency")
    p.add_argument("--oc", action="store_true",
                   help="also time the optical conductivity on the workload's lattice (0-10 eV, 2048 frequencies)")
    p.add_argument("--oc-steps", type=int, default=256)
    p.add_argument("--requests", type=int, default=512)
    p.add_argument("--forms", action="store_true",
                   help="dense workloads: time QE, EC, OC, DP and CD in their sequential and concurrent forms")
    p.add_argument("--forms-steps", type=int, default=512)
    p.add_argument("--seq-steps", type=int, default=0,
                   help="dense workloads: N_t of the D_H sweep against the sequential form (0 = the workload's)")
    p.add_argument("--log2-max-sites", type=int, default=24)
    p.add_argument("--no-serving", action="store_true", help="skip the serving leg of the default line")
    p.add_argument("--serving-requests", type=int, default=512,
                   help="requests of the serving leg (reduced to fit --serving-budget-s, stated in the line)")
    p.add_argument("--serving-budget-s", type=float, default=150.0)
    p.add_argument("--no-c128", action="store_true", help="state-based workloads: complex64 only")
    p.add_argument("--no-state-based", action="store_true",
                   help="skip the time-block leg (vacancy graphene 4096^2) of the default line")
    p.add_argument("--no-largest", action="store_true",
                   help="skip the 1.015e9-site honeycomb leg (S = 4, M = 8192) of the default line")
    p.add_argument("--prof-steps", type=int, default=2,
                   help="steps of the separate profiled pass that times the dominant kernel")
    p.add_argument("--load", type=float, default=0.8, help="arrival rate as a fraction of measured capacity")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(pg, x: float, device=None) -> float:
    """Max of x over the ranks of the default process group (identity without one)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling: fixed units per rank)."""
    return world * units_per_rank / max_seconds


# ---------------------------------------------------------------- clocks during the timed region
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [v.strip() for v in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for k, name in enumerate(names):
                    if parts[5 + k].lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle timing (CPU)
ORACLE_SAMPLE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import lattice as L, propagate as P
kind, dims, t, W, vac, seed, seconds, reps = {kind}, {dims}, {t}, {W}, {vac}, {seed}, {seconds}, {reps}
lat = L.build_lattice(kind, dims, t=t, W=W, vacancy_frac=vac, seed=seed, cutoff={cutoff}, decay={decay})
psi = P.random_phase_states(lat, 1, 1)[0]
t0 = time.perf_counter(); P.moments(lat, psi, psi, 4); one = (time.perf_counter() - t0) / 4
k = int(max(4, min(4096, seconds / max(one, 1e-6))))
out = []
for _ in range(reps):
    t0 = time.perf_counter(); P.moments(lat, psi, psi, k); dt = time.perf_counter() - t0
    out.append(dict(steps=k, seconds=dt, site_updates=k * lat.n))
print(json.dumps(out))
"""


# the same sample, one process per host core, each starting its timed loop once every process
# has built its lattice (a file barrier), so that the loops overlap
ORACLE_SAMPLE_SYNC = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import lattice as L, propagate as P
lat = L.build_lattice({kind}, {dims}, t={t}, W={W}, vacancy_frac={vac}, seed={seed}, cutoff={cutoff}, decay={decay})
psi = P.random_phase_states(lat, 1 + {rank}, 1)[0]
P.moments(lat, psi, psi, 4)
open(os.path.join({sync!r}, "ready{rank}"), "w").close()
while not os.path.exists(os.path.join({sync!r}, "go")):
    time.sleep(0.01)
t0 = time.perf_counter(); k = 0; n = 0
while time.perf_counter() - t0 < {seconds}:
    P.moments(lat, psi, psi, 16); k += 16
dt = time.perf_counter() - t0
print(json.dumps(dict(steps=k, seconds=dt, site_updates=k * lat.n)))
"""


def oracle_sample_all_cores(work: wl.Workload, seconds: float, max_procs: int = 16):
    """The oracle on every host core at once: one single-threaded process per core."""
    spec = work.lattice
    nproc = max(1, min(os.cpu_count() or 1, max_procs))
    sync = tempfile.mkdtemp()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = []
    for rank in range(nproc):
        code = ORACLE_SAMPLE_SYNC.format(root=ROOT, kind=spec.kind, dims=oracle_lattice_dims(spec), t=spec.t, W=spec.W,
                                         vac=spec.vacancy_frac, seed=spec.seed, seconds=seconds, rank=rank, sync=sync,
                                         cutoff=spec.cutoff, decay=spec.decay)
        procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True, env=env))
    deadline = time.time() + 600
    while sum(os.path.exists(os.path.join(sync, f"ready{r}")) for r in range(nproc)) < nproc:
        if time.time() > deadline or any(p.poll() not in (None, 0) for p in procs):
            for p in procs:
                p.kill()
            raise RuntimeError("oracle processes did not start")
        time.sleep(0.05)
    open(os.path.join(sync, "go"), "w").close()
    res = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(err[-1000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    su = sum(r["site_updates"] for r in res)
    wall = max(r["seconds"] for r in res)
    dims = oracle_lattice_dims(spec)
    return {"value": su / wall, "unit": "site-updates/s", "cores": nproc, "kind": "oracle",
            "sample": f"FP64 oracle (numpy/scipy CSR matvec), {nproc} single-threaded processes at once (one per "
                      f"host core), each timing plain Chebyshev steps of one state for {seconds:.0f} s on the "
                      f"{'x'.join(str(d) for d in dims if d > 1)} lattice; rate = all site-updates / the longest loop"}


ORACLE_MAX_SITES = 1 << 25  # larger lattices are sampled on a 2^24-site lattice of the same kind


def oracle_lattice_dims(spec) -> tuple:
    """The lattice the oracle is timed on: the workload's own, or a 2^24-site one of the same kind
    when the workload's would not fit the host (the method is O(N), so the rate carries over).
    Long-range lattices: a 46x46-cell sample (the oracle builds H by brute force over site pairs)."""
    if spec.cutoff > 0:
        return (46, 46, 1)
    if spec.n_full <= ORACLE_MAX_SITES:
        return tuple(spec.L)
    if spec.kind == wl.HONEYCOMB:
        return (2896, 2896, 1)
    if spec.kind == wl.SQUARE:
        return (4096, 4096, 1)
    return (256, 256, 256)


def oracle_sample(work: wl.Workload, seconds: float, reps: int = 1):
    spec = work.lattice
    code = ORACLE_SAMPLE.format(root=ROOT, kind=spec.kind, dims=oracle_lattice_dims(spec), t=spec.t, W=spec.W,
                                vac=spec.vacancy_frac, seed=spec.seed, seconds=seconds, reps=reps,
                                cutoff=spec.cutoff, decay=spec.decay)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_obj(work: wl.Workload, samples):
    su = sum(s["site_updates"] for s in samples)
    sec = sum(s["seconds"] for s in samples)
    dims = oracle_lattice_dims(work.lattice)
    where = (f"the full {wl.KIND_NAMES[work.lattice.kind]} {dims[0]}x{dims[1]} lattice ({work.lattice.n_full} sites)"
             if dims == tuple(work.lattice.L) else
             f"a {wl.KIND_NAMES[work.lattice.kind]} {dims[0]}x{dims[1]} lattice with the same long-range hopping "
             f"(cutoff {work.lattice.cutoff}; the oracle builds H by brute force over site pairs)"
             if work.lattice.cutoff > 0 else
             f"a {wl.KIND_NAMES[work.lattice.kind]} {'x'.join(str(d) for d in dims if d > 1)} lattice of the same "
             f"parameters (the {work.lattice.n_full}-site lattice does not fit the host; O(N) method)")
    return {"value": su / sec, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle (numpy/scipy CSR matvec), 1 state, {samples[0]['steps']} plain Chebyshev "
                      f"steps per sample on {where}, {len(samples)} sample(s), {sec:.1f} s"}


# ---------------------------------------------------------------- roofline inputs
def measured_hbm_peak():
    try:
        with open(PEAKS) as f:
            v = json.load(f).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(kernel_key: str) -> str:
    family = kernel_key.split("/")[0].rstrip("0123456789")
    h = hashlib.sha256()
    for name in KERNEL_SRCS[family]:
        with open(os.path.join(ROOT, "paper_2510_17432_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    try:
        with open(TRAFFIC) as f:
            rec = json.load(f)
        ent = rec.get(kernel_key)
        if ent and ent.get("source_sha256") == kernel_source_hash(kernel_key):
            return float(ent["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


# ---------------------------------------------------------------- reference arm
def run_reference(args, work):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = []
    per_step = max(2.0, min(10.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(work, per_step / 4)
    samples = oracle_sample(work, per_step, reps=args.steps)
    for s in samples:
        steps.append(s)
    su = sum(s["site_updates"] for s in steps)
    sec = sum(s["seconds"] for s in steps)
    value = su / sec
    cpu = cpu_baseline_obj(work, steps)
    print(json.dumps({
        "impl": "reference", "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sec / len(steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox random-phase state)",
        "config": {"workload": work.name, "sites": work.lattice.n_full, "states_per_sample": 1,
                   "form": "plain Chebyshev recurrence (oracle)"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, work):
    import torch
    from paper_2510_17432_gb300 import capi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    ctx = capi.tbpm_create(local)
    capi.tbpm_set_fusion(ctx, args.fusion)
    spec = work.lattice
    desc = capi.lattice_desc(spec.kind, spec.L, t=spec.t, W=spec.W, vacancy_frac=spec.vacancy_frac,
                             seed=spec.seed, pbc=spec.pbc, path=spec.path)
    lat0 = capi.tbpm_lattice_create(ctx, desc)
    info = capi.tbpm_lattice_info(lat0)
    capi.tbpm_lattice_destroy(lat0)
    S, M, nE = work.n_states, work.n_moments, work.n_energies
    E = wl.uniform_energy_grid(nE, info.H0 - info.half_width, info.H0 + info.half_width)
    recon = capi.RECON_TENSOR if args.recon == "tensor" else capi.RECON_FP64
    prec = work.precision
    elem = 8 if prec == capi.C64 else 16
    req = capi.request(n_states=S, precision=prec, form=capi.CONCURRENT_M, n_moments=M,
                       state_seed=1 + 1000 * rank, dos_method=capi.DOS_JACKSON, recon=recon)
    dev = torch.device("cuda", local)
    d_E = torch.tensor(E, device=dev, dtype=torch.float64)
    d_D = torch.empty((S, nE), device=dev, dtype=torch.float64)
    torch.cuda.synchronize()
    stream = torch.cuda.ExternalStream(capi.tbpm_stream(ctx), device=dev)
    site_updates = (M // 2) * info.n_sites * S

    def step_device():
        lat = capi.tbpm_lattice_create(ctx, desc)
        capi.tbpm_dos_device(ctx, lat, req, d_E, nE, d_D)
        capi.tbpm_lattice_destroy(lat)

    def barrier():
        torch.cuda.synchronize()
        capi.tbpm_sync(ctx)
        if pg is not None:
            pg.barrier()

    for _ in range(args.warmup):
        step_device()
    barrier()

    # timed region: the product's own configuration (CUDA graphs on, no phase events)
    clocks = Clocks(local)
    clocks.start()
    launches0 = capi.tbpm_launch_count(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        step_device()
    ev1.record(stream)
    barrier()
    dev_ms = ev0.elapsed_time(ev1)
    launches = capi.tbpm_launch_count(ctx) - launches0
    clk = clocks.stop()
    dev_ms = reduce_max(pg, dev_ms, dev)
    ms_per_step = dev_ms / args.steps
    value = whole_job_rate(site_updates, world, ms_per_step / 1e3)

    # separate profiled pass (phase events on the library stream; graphs off while profiling):
    # the dominant kernel's average launch time and the phase shares of a step
    prof_steps = max(1, args.prof_steps)
    capi.tbpm_profile(ctx, True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    pe0.record(stream)
    for _ in range(prof_steps):
        step_device()
    pe1.record(stream)
    barrier()
    prof_ms = pe0.elapsed_time(pe1)
    prof = capi.tbpm_profile_read(ctx)
    capi.tbpm_profile(ctx, False)

    # parity of this run's output against the oracle is covered by the tests; sanity here
    D = d_D.cpu().numpy()
    assert np.all(np.isfinite(D))

    # ---- end to end through the public API with pinned host buffers
    hE = torch.tensor(E, dtype=torch.float64).pin_memory()
    hD = torch.empty((S, nE), dtype=torch.float64).pin_memory()
    hE_np, hD_np = hE.numpy(), hD.numpy()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lat = capi.tbpm_lattice_create(ctx, desc)
        capi.tbpm_dos(ctx, lat, req, hE_np, hD_np)
        capi.tbpm_lattice_destroy(lat)
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = reduce_max(pg, e2e_s, dev)
    e2e = {"value": whole_job_rate(site_updates, world, e2e_s), "unit": "site-updates/s",
           "h2d_bytes_per_step": int(hE.numel() * 8 + 72), "d2h_bytes_per_step": int(hD.numel() * 8)}

    # ---- roofline of the dominant kernel, from the profiled pass's events.  Unfused one-step
    # pass: 24 B per site-update (read phi_n, read phi_{n-1}, write phi_{n+1}, complex64) + 4 B
    # per site of D_i with disorder.  Fused K-step pass: each state block crosses HBM four times
    # per launch (read phi_{n-1}, phi_n; write phi_{n+K-1}, phi_{n+K}) + D_i once: those are the
    # launch's algorithmic bytes and `frac` is an HBM fraction; the 24 B-per-site-update figure
    # of the same launch is reported beside it as frac_unfused_equiv.
    diag_bytes = (elem / 2) * info.n_sites if spec.W != 0.0 else 0.0
    per_site_step = 3.0 * elem * info.n_sites * S + diag_bytes
    fused_launch = prof["fused_launches"] > 0
    if fused_launch:
        steps_per_launch = FUSION_STEPS[args.fusion]
        kname = FUSION_KERNELS[args.fusion]
        per_launch_ms = prof["fused_ms"] / prof["fused_launches"]
        traffic_key = (f"k_fused_cols{steps_per_launch}/{work.name}" if args.fusion in (1, 2)
                       else f"{FUSION_TRAFFIC_FAMILY.get(args.fusion, 'k_fused_rows')}{steps_per_launch}/{work.name}")
        bytes_per_launch = 4.0 * elem * info.n_sites * S + diag_bytes
        bytes_model = ("fused K-step pass: 4 state-block crossings per launch (read phi_{n-1}, phi_n; write "
                       "phi_{n+K-1}, phi_{n+K}) of N x S x 8 B" + (" + D_i 4 B per site" if diag_bytes else ""))
    else:
        steps_per_launch = 1
        kname = (f"k_moment_stencil<{wl.KIND_NAMES[spec.kind]}, "
                 + ("complex64 x2 per thread>" if prec == capi.C64 and S >= 2 else
                    "complex64 x1 per thread>" if prec == capi.C64 else "complex128>"))
        per_launch_ms = prof["recurrence_ms"] / max(1, prof["recurrence_launches"])
        traffic_key = f"k_moment_stencil/{work.name}"
        bytes_per_launch = per_site_step
        bytes_model = "one-step pass: 24 B per site-update (complex64) + D_i 4 B per site"
    unfused_equiv = per_site_step * steps_per_launch
    achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    traffic = kernel_traffic(traffic_key)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind, "kernel": kname,
                "algorithmic_bytes_per_launch": bytes_per_launch, "bytes_model": bytes_model,
                "avg_launch_us": per_launch_ms * 1e3,
                "site_updates_per_launch": steps_per_launch * info.n_sites * S,
                "frac_unfused_equiv": unfused_equiv / (per_launch_ms / 1e3) / 1e9 / peak,
                "timing": f"CUDA events around the moment passes on the library stream, separate profiled pass "
                          f"of {prof_steps} step(s) after the timed region",
                "recurrence_share_of_step": prof["recurrence_ms"] / prof_ms}
    if traffic:
        roofline["dram_gbs"] = traffic / (per_launch_ms / 1e3) / 1e9
        roofline["dram_frac"] = roofline["dram_gbs"] / peak
        roofline["traffic_over_algorithmic"] = traffic / bytes_per_launch

    recon_ms = prof["recon_ms"] / prof_steps
    Mp = (M + 63) // 64 * 64
    rows_pad = (nE + 127) // 128 * 128
    NP = 16 if 3 * S <= 16 else (32 if 3 * S <= 32 else 48)
    mma_flops = 2.0 * rows_pad * 3 * Mp * NP * (1 if S <= 16 else 2)
    recon = {"ms_per_step": recon_ms, "launches_per_step": prof["recon_launches"] / prof_steps,
             "path": args.recon,
             "mma_tflops": (mma_flops / (recon_ms / 1e3) / 1e12) if args.recon == "tensor" and recon_ms > 0 else None}
    out = {
        "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == capi.C64 else "f64",
        "data": "synthetic (seeded Philox random-phase states on a "
                + ("clean " if spec.W == 0 else f"disordered (W={spec.W}) ") + f"{wl.KIND_NAMES[spec.kind]} lattice)",
        "config": {"workload": work.name, "sites": info.n_sites, "states": S, "moments": M, "energies": nE,
                   "form": "concurrent moment-based, cost-halving (M/2 matrix applications)",
                   "precision": "complex64 states, FP64 reductions" if prec == capi.C64 else "complex128",
                   "reconstruction": args.recon, "fusion_mode": args.fusion, "l2": "inputs larger than L2 (2 state blocks of "
                   f"{info.n_sites * S * 8 / 1e6:.0f} MB)", "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "reconstruction": recon,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }

    # ---- optical conductivity on the same lattice (Fermi-Dirac filtered pair states, time blocks)
    if args.oc and rank == 0:
        lat = capi.tbpm_lattice_create(ctx, desc)
        Nt, nw = args.oc_steps, 2048
        req_oc = capi.request(n_states=S, precision=capi.C64, form=capi.CONCURRENT_S, n_steps=Nt, state_seed=1,
                              window=capi.WINDOW_HANN)
        sig = np.zeros((S, nw), np.complex128)
        mu_f, kT = info.H0, 0.1
        c0 = capi.tbpm_launch_count(ctx)
        t0 = time.perf_counter()
        capi.tbpm_optical_conductivity(ctx, lat, req_oc, 0, 0, mu_f, kT, 10.0, nw, None, sig)
        wall = time.perf_counter() - t0
        capi.tbpm_lattice_destroy(lat)
        out["optical_conductivity"] = {
            "sites": info.n_sites, "states": S, "n_steps": Nt, "tau": "pi/2", "frequencies": nw,
            "omega_max_eV": 10.0, "mu": mu_f, "kT": kT, "form": "time blocks (b autotuned), Hann window",
            "wall_s": wall, "launches": capi.tbpm_launch_count(ctx) - c0,
            "finite": bool(np.all(np.isfinite(sig))), "re_sigma_at_2_7eV": float(np.mean(sig[:, int(2.7 / 10 * 2047)].real))}

    # ---- sequential form on the same GPU: wall time per converged spectrum
    if not args.no_sequential and rank == 0 and work.n_steps:
        Nt = work.n_steps
        Ef = wl.uniform_energy_grid(512, info.H0 - info.half_width, info.H0 + info.half_width)
        res = {}
        for name, form in (("concurrent_m", capi.CONCURRENT_M), ("sequential", capi.SEQUENTIAL)):
            r = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, state_seed=1,
                             dos_method=capi.DOS_FOURIER, window=capi.WINDOW_HANN)
            Dout = np.zeros((S, Ef.size))
            lat = capi.tbpm_lattice_create(ctx, desc)
            c0 = capi.tbpm_launch_count(ctx)
            t0 = time.perf_counter()
            capi.tbpm_dos(ctx, lat, r, Ef, Dout)
            res[name] = (time.perf_counter() - t0, capi.tbpm_launch_count(ctx) - c0, Dout)
            capi.tbpm_lattice_destroy(lat)
        Ntrunc = capi.tbpm_truncation_order(math.pi)
        Mtot = capi.tbpm_truncation_order(Nt * math.pi)
        seq_su = Nt * (Ntrunc - 1) * info.n_sites * S
        conc_su = (Mtot + (Mtot & 1)) // 2 * info.n_sites * S
        diff = float(np.max(np.abs(res["concurrent_m"][2] - res["sequential"][2])) /
                     np.max(np.abs(res["sequential"][2])))
        block = float(info.n_sites) * S * elem
        fused = args.fusion in FUSION_STEPS and FUSION_STEPS[args.fusion] == 4 and spec.kind == wl.HONEYCOMB
        conc_blocks = concurrent_m_blocks(Mtot, fused)
        seq_blocks = Nt * sequential_step_blocks(Ntrunc, fused)
        peak, _ = measured_hbm_peak()
        out["sequential"] = {
            "n_steps": Nt, "tau": "pi", "dos": "Hann-windowed Fourier DOS on 512 energies",
            "wall_s_concurrent": res["concurrent_m"][0], "wall_s_sequential": res["sequential"][0],
            "speedup_wall": res["sequential"][0] / res["concurrent_m"][0],
            "matrix_applications_concurrent": conc_su // (info.n_sites * S),
            "matrix_applications_sequential": seq_su // (info.n_sites * S),
            "speedup_matrix_applications": seq_su / conc_su,
            "state_block_crossings_concurrent": conc_blocks, "state_block_crossings_sequential": seq_blocks,
            "speedup_hbm_bytes": seq_blocks / conc_blocks,
            "hbm_frac_concurrent": conc_blocks * block / res["concurrent_m"][0] / 1e9 / peak,
            "hbm_frac_sequential": seq_blocks * block / res["sequential"][0] / 1e9 / peak,
            "bytes_model": "state blocks of N x S x 8 B crossing HBM: concurrent = moment passes (4 per "
                           "four-step pass, 3 per one-step pass); sequential = per time step the buffered "
                           "time block of the library (copy, first step, four-term window passes writing 4 "
                           "slots, one-step passes, one flush reading every term, <psi|psi(t)>, carry)",
            "site_updates_per_s_sequential": seq_su / res["sequential"][0],
            "site_updates_per_s_concurrent": conc_su / res["concurrent_m"][0],
            "max_rel_dos_difference": diff}

    if rank == 0 and not args.no_serving and work is wl.GRAPHENE_2048:
        out["serving"] = serving_leg(capi, ctx, args, args.serving_requests, args.serving_budget_s)

    if rank == 0 and not args.no_largest and work is wl.GRAPHENE_2048:
        try:
            out["largest_config"] = largest_leg(capi, ctx, args)
        except Exception as exc:  # the headline number stands; say why this leg is missing
            out["largest_config"] = {"workload": wl.GRAPHENE_22528.name, "failed": f"{exc!r}"[:300]}

    if rank == 0 and not args.no_state_based and work is wl.GRAPHENE_2048:
        try:
            out["state_based"] = state_based_leg(capi, ctx, args)
        except Exception as exc:
            out["state_based"] = {"workload": wl.GRAPHENE_4096_VAC.name, "failed": f"{exc!r}"[:300]}

    if rank == 0 and not args.no_cpu and world == 1:
        try:
            out["cpu_baseline"] = cpu_baseline_obj(work, oracle_sample(work, args.cpu_seconds))
        except Exception as exc:  # the GPU number stands; say why the baseline is missing
            out["cpu_baseline"] = {"value": None, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
                                   "sample": f"failed: {exc!r}"[:300]}
        try:
            out["cpu_baseline_all_cores"] = oracle_sample_all_cores(work, min(10.0, args.cpu_seconds))
        except Exception as exc:
            out["cpu_baseline_all_cores"] = {"value": None, "unit": "site-updates/s", "kind": "oracle",
                                             "sample": f"failed: {exc!r}"[:300]}
    elif rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = None

    capi.tbpm_destroy(ctx)
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


# ---------------------------------------------------------------- byte models of the two forms
def concurrent_m_blocks(n_moments: int, fused: bool) -> float:
    """State-block crossings of the moment pass for n_moments moments (cost halving: M/2 steps):
    initialisation writes phi_0, the first one-step pass reads it and writes phi_1 (with the
    moments), then four-step passes (read 2, write 2) where the register sweep runs, and one-step
    passes (read phi_n, phi_{n-1}, write phi_{n+1}) for the rest."""
    steps = (n_moments + (n_moments & 1)) // 2
    blocks = 1 + 2
    n = 1
    if fused:
        while n + 4 <= steps:
            blocks += 4
            n += 4
    return blocks + 3 * (steps - n)


def sequential_step_blocks(n_terms: int, fused: bool) -> float:
    """State-block crossings of one sequential time step as the library buffers it (b = 1):
    clear the accumulator, copy psi(t) into the first slot, the first term H~ phi_0, four-term
    window passes (read 2, write 4) while four terms fit, one-step passes (read 2, write 1) for
    the rest, one flush (read every term, read and write the accumulator), <psi|psi(t)> (2) and
    the copy of psi(t) for the next step (2)."""
    blocks = 1 + 2 + 2
    n = 2
    if fused:
        while n + 3 < n_terms:
            blocks += 6
            n += 4
    blocks += 3 * (n_terms - n)
    return blocks + n_terms + 2 + 2 + 2


# ---------------------------------------------------------------- state-based correlation (vacancy lattices)
def state_based_schedule(n_steps: int, b: int, tau: float, trunc) -> tuple:
    """Passes of the time-block form in the library's order: for every block of bb <= b steps,
    Chebyshev terms n = 0..N_b-1 with the accumulators of times j whose N((j+1) tau) > n open.
    Returns (matrix applications, [(open accumulators, spmv?, first?) per pass], block count)."""
    passes, apps, blocks = [], 0, 0
    start = 0
    while start < n_steps:
        bb = min(b, n_steps - start)
        nper = [trunc((j + 1) * tau) for j in range(bb)]
        Nb = max(nper)
        for n in range(Nb):
            opened = sum(1 for j in range(bb) if nper[j] > n)
            spmv = n < Nb - 1
            passes.append((opened, spmv, n == 0))
            apps += spmv
        blocks += 1
        start += bb
    return apps, passes, blocks


def state_based_bytes(passes, blocks, n_sites, S, elem, z, diag_bytes, n_steps, corr=True) -> float:
    """Algorithmic bytes of the time-block passes: per pass read phi_n, and with a matrix
    application read phi_{n-1} (not on the first term), write phi_{n+1}, the ELL lists (4z B per
    site) and D_i; per open accumulator write (first term) or read + write; per time step one read
    of psi for <psi|psi(t)>; per block the copy of its last state."""
    st = float(n_sites) * S * elem
    total = 0.0
    for opened, spmv, first in passes:
        total += st
        if spmv:
            total += st + (0.0 if first else st) + 4.0 * z * n_sites + diag_bytes * n_sites
        total += opened * st * (1.0 if first else 2.0)
    total += blocks * 2.0 * st
    if corr:
        total += n_steps * st
    return total


def state_based_bytes_buffered(n_steps: int, b: int, tau: float, trunc, n_sites, S, elem, z, diag_bytes,
                               T: int = 32, corr=True) -> float:
    """Bytes moved by the buffered time blocks (b >= 2): per block the accumulators are cleared,
    phi_0 copied into the buffer; every recurrence step reads phi_n, phi_{n-1} (not the first),
    the ELL lists and D_i and writes phi_{n+1} into a slot; every window of <= T terms is read
    once per 16 accumulators and each accumulator read and written once; two slots are carried
    to the next window; <psi|acc_j> reads psi and the accumulators; the last state is copied."""
    st = float(n_sites) * S * elem
    total = 0.0
    start = 0
    while start < n_steps:
        bb = min(b, n_steps - start)
        Nb = max(trunc((j + 1) * tau) for j in range(bb))
        tiles = (bb + 15) // 16
        total += bb * st + 2 * st
        for n in range(1, Nb):
            total += (2 if n == 1 else 3) * st + 4.0 * z * n_sites + diag_bytes * n_sites
        windows = (Nb + T - 1) // T
        total += Nb * st * tiles + windows * 2 * bb * st + (windows - 1) * 4 * st
        if corr:
            total += st * tiles + bb * st
        total += 2 * st
        start += bb
    return total


def time_block_forms(capi, ctx, lat, spec, N, S, Nt, prec, warmup, reps, peak, seed=1, seq_warmup=1) -> dict:
    """C(t_j), j <= Nt, at tau~ = pi through the state-based time-block form (b autotuned from
    measured pass costs) and the sequential form on one lattice in one precision: seconds per
    call (CUDA events on the library stream, inputs resident), matrix applications, launches,
    site-updates/s, HBM fraction by the byte model, and the largest relative C difference."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.ExternalStream(capi.tbpm_stream(ctx), device=dev)
    elem, dbytes = (8, 4) if prec == capi.C64 else (16, 8)
    tau = math.pi
    trunc = capi.tbpm_truncation_order
    z = wl.COORDINATION[spec.kind]

    def timed_corr(form, b, n_warm, n_reps):
        req = capi.request(n_states=S, precision=prec, form=form, n_steps=Nt, time_block=b, state_seed=seed)
        d_C = torch.empty((max(S, 1), Nt + 1, 2), device=dev, dtype=torch.float64)
        for _ in range(n_warm):
            capi.tbpm_correlation_device(ctx, lat, req, d_C)
        capi.tbpm_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = capi.tbpm_launch_count(ctx)
        e0.record(stream)
        for _ in range(n_reps):
            capi.tbpm_correlation_device(ctx, lat, req, d_C)
        e1.record(stream)
        capi.tbpm_sync(ctx)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / n_reps, (capi.tbpm_launch_count(ctx) - l0) // n_reps, d_C.cpu().numpy()

    b_opt, t_a, t_x = capi.tbpm_block_autotune(ctx, lat, capi.request(n_states=S, precision=prec, form=2,
                                                                        n_steps=Nt, state_seed=seed), Nt)
    res = {}
    for name, form, b in (("concurrent_s", capi.CONCURRENT_S, b_opt), ("sequential", capi.SEQUENTIAL, 1)):
        n_reps = reps if name == "concurrent_s" else 1
        n_warm = (warmup if n_reps > 1 else 1) if name == "concurrent_s" else seq_warmup
        sec, launches, C = timed_corr(form, b, n_warm, n_reps)
        apps, passes, blocks = state_based_schedule(Nt, b, tau, trunc)
        if b >= 2:  # buffered time blocks (the library's default for b >= 2)
            alg = state_based_bytes_buffered(Nt, b, tau, trunc, N, S, elem, z, dbytes if spec.W != 0 else 0)
        else:
            alg = state_based_bytes(passes, blocks, N, S, elem, z, dbytes if spec.W != 0 else 0, Nt)
        res[name] = {"b": b, "seconds": sec, "reps": n_reps, "matrix_applications": apps, "launches": launches,
                     "site_updates_per_s": apps * N * S / sec, "algorithmic_gbs": alg / sec / 1e9,
                     "frac_of_hbm": alg / sec / 1e9 / peak, "C": C}
    diff = float(np.max(np.abs(res["concurrent_s"]["C"] - res["sequential"]["C"])) /
                 np.max(np.abs(res["sequential"]["C"])))
    for r in res.values():
        r.pop("C")
    return {"t_amxsy_ms": t_a, "t_axpy_ms": t_x, "b_opt": b_opt, **res,
            "speedup_wall": res["sequential"]["seconds"] / res["concurrent_s"]["seconds"],
            "max_rel_correlation_difference": diff}


def state_based_leg(capi, ctx, args) -> dict:
    """Time evolution on graphene 4096 x 4096 with 1 % vacancies and V in [-1, 1] eV (33.2M sites
    on the ELL path), one complex64 state, Nt = 2048 steps at the Nyquist step tau~ = pi: the
    state-based time-block form against the sequential form, one timed call each."""
    work = wl.GRAPHENE_4096_VAC
    spec = work.lattice
    desc = capi.lattice_desc(spec.kind, spec.L, t=spec.t, W=spec.W, vacancy_frac=spec.vacancy_frac,
                             seed=spec.seed, pbc=spec.pbc, path=spec.path)
    t0 = time.perf_counter()
    lat = capi.tbpm_lattice_create(ctx, desc)
    capi.tbpm_sync(ctx)
    build_s = time.perf_counter() - t0
    try:
        info = capi.tbpm_lattice_info(lat)
        peak, peak_kind = measured_hbm_peak()
        import torch
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        forms = time_block_forms(capi, ctx, lat, spec, info.n_sites, work.n_states, work.n_steps, capi.C64,
                                 1, 1, peak, seed=1, seq_warmup=0)
        clk = clocks.stop()
    finally:
        capi.tbpm_lattice_destroy(lat)
    return {"workload": work.name, "sites": info.n_sites, "states": work.n_states, "n_steps": work.n_steps,
            "tau": "pi", "precision": "c64", "path": "ELL (vacancies)", "lattice_build_s": build_s,
            "peak_gbs": peak, "peak_source": peak_kind, **forms, "clocks": clk,
            "timing": "CUDA events on the library stream; one warm-up call of the time-block form, none "
                      "of the sequential form (same kernels)"}


def run_state_based(args, work):
    import torch
    from paper_2510_17432_gb300 import capi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    dev = torch.device("cuda", local)
    ctx = capi.tbpm_create(local)
    spec = work.lattice
    desc = capi.lattice_desc(spec.kind, spec.L, t=spec.t, W=spec.W, vacancy_frac=spec.vacancy_frac,
                             seed=spec.seed, pbc=spec.pbc, path=spec.path)
    lat = capi.tbpm_lattice_create(ctx, desc)
    info = capi.tbpm_lattice_info(lat)
    N, S, Nt = info.n_sites, work.n_states, work.n_steps

    out_forms = {}
    peak, peak_kind = measured_hbm_peak()
    clocks = Clocks(local)
    clocks.start()
    for prec in ((capi.C64,) if args.no_c128 else (capi.C64, capi.C128)):
        reps = {capi.C64: args.steps, capi.C128: 1}
        out_forms["c64" if prec == capi.C64 else "c128"] = time_block_forms(
            capi, ctx, lat, spec, N, S, Nt, prec, args.warmup, reps[prec], peak, seed=1 + rank)
    clk = clocks.stop()

    # DC conductivity and quasi-eigenstates at the workload's energies (complex64), all three EC forms
    ec = {}
    if work.n_energies and not args.no_sequential:
        E = wl.uniform_energy_grid(work.n_energies, info.H0 - 0.8 * info.half_width, info.H0 + 0.8 * info.half_width)
        sig = {}
        for name, form in (("ec_concurrent_m", capi.CONCURRENT_M), ("ec_concurrent_s", capi.CONCURRENT_S),
                           ("ec_sequential", capi.SEQUENTIAL)):
            sg = np.zeros((S, E.size))
            t0 = time.perf_counter()
            capi.tbpm_conductivity(ctx, lat, capi.request(n_states=S, precision=capi.C64, form=form, n_steps=Nt,
                                                          state_seed=1), 0, E, None, sg)
            ec[name + "_wall_s"] = time.perf_counter() - t0
            sig[name] = sg
        ref = sig["ec_sequential"]
        ec["energies"] = int(E.size)
        ec["quasi_eigenstates"] = "energy-based form inside every EC call (N_E <= 200)"
        ec["max_rel_sigma_difference_m_vs_seq"] = float(np.max(np.abs(sig["ec_concurrent_m"] - ref)) /
                                                        np.max(np.abs(ref)))
        ec["max_rel_sigma_difference_s_vs_seq"] = float(np.max(np.abs(sig["ec_concurrent_s"] - ref)) /
                                                        np.max(np.abs(ref)))
    c64 = out_forms["c64"]
    value = whole_job_rate(c64["concurrent_s"]["site_updates_per_s"], world, 1.0)
    roofline = {"bound": "hbm", "achieved": c64["concurrent_s"]["algorithmic_gbs"], "peak": peak, "unit": "GB/s",
                "frac": c64["concurrent_s"]["frac_of_hbm"], "traffic": None, "peak_source": peak_kind,
                "kernel": ("k_ell_step (ELL recurrence into buffer slots) + k_block_flush_c64 (packed flush), complex64"
                           if c64["concurrent_s"]["b"] >= 2 else "k_accum_step (ELL, complex64, time-block accumulation)"),
                "bytes_model": ("buffered blocks: per step phi_n, phi_{n-1}, phi_{n+1}, 4z B ELL + D_i per site; per "
                                "window of <= 32 terms each slot read once per 16 accumulators and each accumulator "
                                "read and written once; per block clear, copies and one block inner product"
                                if c64["concurrent_s"]["b"] >= 2 else
                                "per pass: phi_n, phi_{n-1}, phi_{n+1}, 4z B ELL + D_i per site, 8 or 16 B per "
                                "open accumulator, psi once per time step, one copy per block")}
    out = {"metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * c64["concurrent_s"]["seconds"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded Philox random-phase state, vacancies and disorder)",
           "config": {"workload": work.name, "sites": N, "states": S, "n_steps": Nt, "tau": "pi",
                      "form": "state-based time blocks (b autotuned from measured pass costs)",
                      "path": "ELL (vacancies)", "l2": f"inputs larger than L2 ({N * S * 8 / 1e6:.0f} MB per state block)",
                      "parallelism": f"replicas x{world}"},
           "roofline": roofline, "forms": out_forms, "conductivity": ec or None,
           "e2e": None, "gpu_launches": c64["concurrent_s"]["launches"], "clocks": clk}
    # end to end through tbpm_correlation (host buffer)
    Ch = np.zeros((S, Nt + 1), np.complex128)
    req = capi.request(n_states=S, precision=capi.C64, form=capi.CONCURRENT_S, n_steps=Nt,
                       time_block=c64["concurrent_s"]["b"], state_seed=1)
    t0 = time.perf_counter()
    capi.tbpm_correlation(ctx, lat, req, Ch)
    e2e_s = reduce_max(pg, time.perf_counter() - t0, dev)
    out["e2e"] = {"value": whole_job_rate(c64["concurrent_s"]["matrix_applications"] * N * S, world, e2e_s),
                  "unit": "site-updates/s", "h2d_bytes_per_step": 72, "d2h_bytes_per_step": int(Ch.nbytes)}
    if rank == 0 and not args.no_cpu and world == 1:
        try:
            out["cpu_baseline"] = cpu_baseline_obj(work, oracle_sample(work, args.cpu_seconds))
        except Exception as exc:
            out["cpu_baseline"] = {"value": None, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
                                   "sample": f"failed: {exc!r}"[:300]}
    capi.tbpm_lattice_destroy(lat)
    capi.tbpm_destroy(ctx)
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


# ---------------------------------------------------------------- serving stream
def request_work(r):
    n = r.lattice.n_full
    return (r.n_moments // 2) * n * r.n_states


def serving_leg(capi, ctx, args, n_requests: int, budget_s: float | None = None) -> dict:
    """The request stream of the serving configuration: Poisson arrivals of DOS / LDOS requests
    (square, honeycomb or simple-cubic lattices, 2^12..2^log2_max sites, W ~ U[0,2]t, M ~ U{256..8192},
    S ~ U{1..16} or LDOS at 32 sites) at `--load` x the capacity measured by a closed-loop probe,
    served by one server (continuous batching into the persistent kernel).  With a time budget the
    stream is cut to the first requests whose work fits it at that rate (stated in the result)."""
    import threading

    E = wl.uniform_energy_grid(1024, -8.2, 8.2)
    recon = capi.RECON_TENSOR if args.recon == "tensor" else capi.RECON_FP64

    def submit(srv, r):
        sp = r.lattice
        desc = capi.lattice_desc(sp.kind, sp.L, t=sp.t, W=sp.W, seed=sp.seed)
        if r.quantity == "ldos":
            req = capi.request(sites=r.sites, precision=capi.C64, n_moments=r.n_moments)
        else:
            req = capi.request(n_states=r.n_states, precision=capi.C64, n_moments=r.n_moments, state_seed=sp.seed)
        return capi.tbpm_submit(srv, desc, req, E)

    # capacity probe: a closed-loop burst of requests from the same distribution
    probe = wl.serving_stream(24, 1.0, seed=wl.REQUEST_SEED + 1, log2_max=args.log2_max_sites)
    srv = capi.tbpm_server_create(ctx, recon=recon)
    t0 = time.perf_counter()
    ts = [submit(srv, r) for r in probe]
    for t, r in zip(ts, probe):
        capi.tbpm_wait(srv, t, np.zeros((r.n_states, E.size)))
    cap_su = sum(request_work(r) for r in probe) / (time.perf_counter() - t0)
    capi.tbpm_server_destroy(srv)

    full = wl.serving_stream(n_requests, 1.0, log2_max=args.log2_max_sites)
    mean_work = sum(request_work(r) for r in full) / len(full)
    rate = args.load * cap_su / mean_work
    stream = wl.serving_stream(n_requests, rate, log2_max=args.log2_max_sites)
    cut = len(stream)
    if budget_s:
        work = 0.0
        for i, r in enumerate(stream):
            work += request_work(r)
            if max(r.arrival_s, work / (args.load * cap_su)) > budget_s:
                cut = max(16, i)
                break
    stream = stream[:cut]
    srv = capi.tbpm_server_create(ctx, recon=recon)
    tickets = [None] * len(stream)
    start = time.perf_counter()

    def submitter():
        for i, r in enumerate(stream):
            delay = start + r.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[i] = submit(srv, r)

    th = threading.Thread(target=submitter)
    th.start()
    lat = []
    for i, r in enumerate(stream):
        while tickets[i] is None:
            time.sleep(0.0005)
        q, run, tot = capi.tbpm_wait(srv, tickets[i], np.zeros((r.n_states, E.size)))
        lat.append(tot / 1e3)
    th.join()
    makespan = time.perf_counter() - start
    stats = capi.tbpm_server_stats(srv)
    capi.tbpm_server_destroy(srv)
    lat = np.array(lat)
    total_su = sum(request_work(r) for r in stream)
    sizes = [r.lattice.n_full for r in stream]
    return {
        "requests": len(stream), "requests_planned": n_requests,
        "cut": (None if cut == n_requests else
                f"first {cut} of the {n_requests} arrivals: their work at {args.load} x capacity fills the "
                f"{budget_s:.0f} s time budget of this leg; same distribution, same arrival process"),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "latency": "submit to DOS copied into the caller's host buffer",
        "throughput_site_updates_per_s": total_su / makespan, "makespan_s": makespan,
        "arrival_rate_per_s": rate, "load": args.load, "capacity_site_updates_per_s": cap_su,
        "sites_min": int(min(sizes)), "sites_max": int(max(sizes)),
        "kernel_launches": stats["launches"], "batched_kernel_gpu_s": stats["gpu_us"] / 1e6,
        "workload": f"Poisson arrivals, square/honeycomb/cubic, 2^12..2^{args.log2_max_sites} sites, W~U[0,2]t, "
                    "M~U{256..8192}, S~U{1..16} or LDOS at 32 sites, complex64, Jackson DOS on 1024 energies",
        "reconstruction": args.recon}


def run_serving(args):
    from paper_2510_17432_gb300 import capi

    rank, world, local = dist_env()
    ctx = capi.tbpm_create(local)
    res = serving_leg(capi, ctx, args, args.requests)
    capi.tbpm_destroy(ctx)
    print(json.dumps({"metric": "serving latency (submit to DOS on host) and throughput", "n_gpus": 1,
                      "dtype": "f32", "data": "synthetic", **res}))


def largest_leg(capi, ctx, args) -> dict:
    """The 1.015e9-site honeycomb (22528 x 22528 cells, V in [-0.5, 0.5] eV, 4 complex64 states,
    8192 moments, Jackson DOS on 8192 energies): one timed spectrum through tbpm_dos_device after
    a short warm-up request on the same lattice."""
    import torch

    work = wl.GRAPHENE_22528
    spec = work.lattice
    desc = capi.lattice_desc(spec.kind, spec.L, t=spec.t, W=spec.W, seed=spec.seed, pbc=spec.pbc, path=spec.path)
    t0 = time.perf_counter()
    lat = capi.tbpm_lattice_create(ctx, desc)
    capi.tbpm_sync(ctx)
    build_s = time.perf_counter() - t0
    info = capi.tbpm_lattice_info(lat)
    S, M, nE = work.n_states, work.n_moments, 8192
    E = wl.uniform_energy_grid(nE, info.H0 - info.half_width, info.H0 + info.half_width)
    dev = torch.device("cuda", torch.cuda.current_device())
    d_E = torch.tensor(E, device=dev, dtype=torch.float64)
    d_D = torch.empty((S, nE), device=dev, dtype=torch.float64)
    recon = capi.RECON_TENSOR if args.recon == "tensor" else capi.RECON_FP64
    warm = capi.request(n_states=S, precision=work.precision, n_moments=64, state_seed=1,
                        dos_method=capi.DOS_JACKSON, recon=recon)
    capi.tbpm_dos_device(ctx, lat, warm, d_E, nE, d_D)
    req = capi.request(n_states=S, precision=work.precision, n_moments=M, state_seed=1,
                       dos_method=capi.DOS_JACKSON, recon=recon)
    stream = torch.cuda.ExternalStream(capi.tbpm_stream(ctx), device=dev)
    capi.tbpm_sync(ctx)
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = capi.tbpm_launch_count(ctx)
    e0.record(stream)
    capi.tbpm_dos_device(ctx, lat, req, d_E, nE, d_D)
    e1.record(stream)
    capi.tbpm_sync(ctx)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = e0.elapsed_time(e1) / 1e3
    D = d_D.cpu().numpy()
    capi.tbpm_lattice_destroy(lat)
    su = (M // 2) * info.n_sites * S
    return {"workload": work.name, "sites": info.n_sites, "states": S, "moments": M, "energies": nE,
            "steps": 1, "warmup": "one 64-moment request on the same lattice",
            "seconds_per_spectrum": sec, "site_updates_per_s": su / sec, "launches": capi.tbpm_launch_count(ctx) - l0,
            "lattice_build_s": build_s, "finite": bool(np.all(np.isfinite(D))), "clocks": clk,
            "timing": "CUDA events on the library stream around one tbpm_dos_device call (graphs on)"}


def dense_desc(capi, spec):
    return capi.lattice_desc(spec.kind, spec.L, t=spec.t, W=spec.W, vacancy_frac=spec.vacancy_frac, seed=spec.seed,
                             pbc=spec.pbc, path=spec.path, cutoff=spec.cutoff, decay=spec.decay)


def dense_forms(capi, ctx, desc, S, Nt):
    """Every quantity of the paper in its sequential and concurrent forms on the dense lattice
    (Secs. IV-VIII measure these speedups on the D_H = 230 sample): wall time per call, same GPU."""
    lat = capi.tbpm_lattice_create(ctx, desc)
    info = capi.tbpm_lattice_info(lat)
    n = info.n_sites
    width = info.E_max - info.E_min
    E = info.H0 + np.array([-0.5, -0.1, 0.2, 0.6]) * width / 2
    mu, kT = info.H0, 0.05 * width / 2
    om = np.linspace(0.0, width, 256)
    res = {"n_steps": Nt, "states": S, "energies": E.size, "kT": kT}

    def timed(fn):
        capi.tbpm_sync(ctx)
        t0 = time.perf_counter()
        fn()
        capi.tbpm_sync(ctx)
        return time.perf_counter() - t0

    def req(form, b=0, tau=0.0):
        return capi.request(n_states=S, precision=capi.C64, form=form, n_steps=Nt, time_block=b, state_seed=1, tau=tau)

    qe = np.zeros((E.size, S, n), np.complex64)
    res["qe"] = {name: timed(lambda f=f: capi.tbpm_quasi_eigenstates(ctx, lat, req(f), E, qe))
                 for name, f in (("sequential", capi.SEQUENTIAL), ("concurrent_s", capi.CONCURRENT_S),
                                 ("concurrent_e", capi.CONCURRENT_E))}
    sig = np.zeros((S, E.size))
    res["ec"] = {name: timed(lambda f=f: capi.tbpm_conductivity(ctx, lat, req(f), 0, E, None, sig))
                 for name, f in (("sequential", capi.SEQUENTIAL), ("concurrent_s", capi.CONCURRENT_S),
                                 ("concurrent_m", capi.CONCURRENT_M))}
    so = np.zeros((S, om.size), np.complex128)
    res["oc"] = {name: timed(lambda f=f: capi.tbpm_optical_conductivity(ctx, lat, req(f), 0, 0, mu, kT, width,
                                                                         om.size, None, so))
                 for name, f in (("sequential", capi.SEQUENTIAL), ("concurrent_s", capi.CONCURRENT_S))}
    res["dp"] = {name: timed(lambda f=f: capi.tbpm_polarization(ctx, lat, req(f), (0.3, 0.1, 0.0), mu, kT, om,
                                                                 None, so))
                 for name, f in (("sequential", capi.SEQUENTIAL), ("concurrent_s", capi.CONCURRENT_S))}
    rho = np.zeros((S, n))
    res["cd"] = {name: timed(lambda f=f: capi.tbpm_charge_density(ctx, lat, req(f), mu, kT, rho))
                 for name, f in (("sequential", capi.SEQUENTIAL), ("concurrent_s", capi.CONCURRENT_S))}
    b_opt, t_amxsy, t_axpy = capi.tbpm_block_autotune(ctx, lat, req(capi.CONCURRENT_S), Nt)
    res["time_block"] = {"b_opt": b_opt, "t_amxsy_ms": t_amxsy, "t_axpy_ms": t_axpy}
    for q in ("qe", "ec", "oc", "dp", "cd"):
        seq = res[q]["sequential"]
        res[q]["speedup"] = {k: seq / v for k, v in res[q].items() if k != "sequential"}
    capi.tbpm_lattice_destroy(lat)
    return res


def run_dense(args, work):
    """Dense Hamiltonians (long-range hopping, D_H = 61 / 124 / 235; the stand-in for the paper's
    twisted bilayer graphene): the moment-based concurrent DOS over N_t steps of tau~ = pi (the
    paper's DOS-Concurrent-M, Sec. III) is the timed step; the sweep over D_H times it against
    the sequential form on the same GPU (the paper's speedup-vs-D_H benchmark)."""
    import torch
    from paper_2510_17432_gb300 import capi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    dev = torch.device("cuda", local)
    ctx = capi.tbpm_create(local)
    spec = work.lattice
    desc = dense_desc(capi, spec)
    lat = capi.tbpm_lattice_create(ctx, desc)
    info = capi.tbpm_lattice_info(lat)
    S, Nt, nE = work.n_states, work.n_steps, work.n_energies
    E = wl.uniform_energy_grid(nE, info.H0 - info.half_width, info.H0 + info.half_width)
    Mtot = capi.tbpm_truncation_order(Nt * math.pi)
    n_mat = (Mtot + (Mtot & 1)) // 2
    site_updates = n_mat * info.n_sites * S
    req = capi.request(n_states=S, precision=work.precision, form=capi.CONCURRENT_M, n_steps=Nt,
                       state_seed=1 + 1000 * rank, dos_method=capi.DOS_FOURIER, window=capi.WINDOW_HANN)
    d_E = torch.tensor(E, device=dev, dtype=torch.float64)
    d_D = torch.empty((S, nE), device=dev, dtype=torch.float64)
    stream = torch.cuda.ExternalStream(capi.tbpm_stream(ctx), device=dev)

    def step_device():
        capi.tbpm_dos_device(ctx, lat, req, d_E, nE, d_D)

    def barrier():
        torch.cuda.synchronize()
        capi.tbpm_sync(ctx)
        if pg is not None:
            pg.barrier()

    for _ in range(args.warmup):
        step_device()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = capi.tbpm_launch_count(ctx)
    capi.tbpm_profile(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        step_device()
    ev1.record(stream)
    barrier()
    dev_ms = reduce_max(pg, ev0.elapsed_time(ev1), dev)
    prof = capi.tbpm_profile_read(ctx)
    capi.tbpm_profile(ctx, False)
    launches = capi.tbpm_launch_count(ctx) - launches0
    clk = clocks.stop()
    ms_per_step = dev_ms / args.steps
    value = whole_job_rate(site_updates, world, ms_per_step / 1e3)
    assert np.all(np.isfinite(d_D.cpu().numpy()))

    hE = torch.tensor(E, dtype=torch.float64).pin_memory()
    hD = torch.empty((S, nE), dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        capi.tbpm_dos(ctx, lat, req, hE.numpy(), hD.numpy())
    barrier()
    e2e_s = reduce_max(pg, (time.perf_counter() - t0) / args.steps, dev)
    e2e = {"value": whole_job_rate(site_updates, world, e2e_s), "unit": "site-updates/s",
           "h2d_bytes_per_step": int(hE.numel() * 8 + 72), "d2h_bytes_per_step": int(hD.numel() * 8)}

    # roofline of the recurrence pass.  The library reports which kernel carries it.  The tap
    # kernel (clean long-range lattices, complex64, >= 2 states, a tile that fits shared memory)
    # is bound by FP32 FMA issue: 2 FMAs (real weight x complex state) per tap per site-update,
    # against the device's SM count x 128 FP32 lanes x 2 flops x the median SM clock sampled during
    # the timed region.  Otherwise the ELL kernel: HBM-bound on the index lists.
    z = info.coordination
    elem = 8 if work.precision == capi.C64 else 16
    per_launch_ms = prof["recurrence_ms"] / max(1, prof["recurrence_launches"])
    peak, peak_kind = measured_hbm_peak()
    state_bytes = 3.0 * elem * S * info.n_sites
    flops_per_launch = 4.0 * z * info.n_sites * S
    props = torch.cuda.get_device_properties(dev)
    sm_count, lanes = props.multi_processor_count, 128
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    derived_peak = sm_count * lanes * sm_mhz * 1e6 * 2 / 1e12
    fma_scalar, fma_packed = capi.tbpm_fp32_fma_peak(ctx)
    alu_peak = max(fma_scalar, fma_packed)
    pass_kind = capi.tbpm_moment_pass_kind(ctx, lat, req)
    if pass_kind == capi.PASS_TAPS:
        achieved = flops_per_launch / (per_launch_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "traffic": None,
                    "peak_source": "measured: FMA chains on this device (tbpm_fp32_fma_peak), the larger of "
                                   f"scalar {fma_scalar:.1f} and packed f32x2 {fma_packed:.1f} TFLOP/s",
                    "derived_peak_tflops": derived_peak,
                    "derived_peak_source": f"{sm_count} SMs (device) x {lanes} FP32 lanes x 2 flops x {sm_mhz:.0f} MHz "
                                           "(median SM clock sampled during the timed region)",
                    "kernel": f"k_taps_moment<{wl.KIND_NAMES[spec.kind]}> (matrix-free taps, two complex64 states per pack)",
                    "algorithmic_flops_per_launch": flops_per_launch, "avg_launch_us": per_launch_ms * 1e3,
                    "hbm_algorithmic_gbs": state_bytes / (per_launch_ms / 1e3) / 1e9, "hbm_peak_gbs": peak,
                    "recurrence_share_of_step": prof["recurrence_ms"] / dev_ms}
    else:
        bytes_per_launch = state_bytes + 4.0 * z * info.n_sites
        achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": None, "peak_source": peak_kind,
                    "kernel": f"k_moment_step<CSR> (ELL lists + per-slot weights, {wl.KIND_NAMES[spec.kind]})",
                    "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_us": per_launch_ms * 1e3,
                    "fp32_tflops": flops_per_launch / (per_launch_ms / 1e3) / 1e12, "fp32_peak_tflops": alu_peak,
                    "fp32_peak_source": "measured (tbpm_fp32_fma_peak)",
                    "recurrence_share_of_step": prof["recurrence_ms"] / dev_ms}
    out = {
        "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if work.precision == capi.C64 else "f64",
        "data": "synthetic (seeded Philox random-phase states on a clean long-range honeycomb lattice)",
        "config": {"workload": work.name, "sites": info.n_sites, "D_H": z + 1, "states": S, "n_steps": Nt,
                   "moments": Mtot, "matrix_applications": n_mat, "energies": nE,
                   "form": "concurrent moment-based DOS (Hann-windowed Fourier of C(t) from moments)",
                   "l2": "working set larger than L2: two state blocks of %.0f MB each are read and one written "
                         "per launch (L2 129 MB)" % (info.n_sites * S * elem / 1e6),
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
    }
    capi.tbpm_lattice_destroy(lat)

    if rank == 0 and not args.no_sequential:
        sweep = []
        Ef = wl.uniform_energy_grid(512, info.H0 - info.half_width, info.H0 + info.half_width)
        Nseq = args.seq_steps or Nt
        for dh in sorted(wl.DENSE_CUTOFFS):
            w2 = wl.dense_honeycomb(dh, n_states=S, n_steps=Nseq)
            l2 = capi.tbpm_lattice_create(ctx, dense_desc(capi, w2.lattice))
            i2 = capi.tbpm_lattice_info(l2)
            res = {}
            for name, form in (("concurrent_m", capi.CONCURRENT_M), ("sequential", capi.SEQUENTIAL)):
                r = capi.request(n_states=S, precision=work.precision, form=form, n_steps=Nseq, state_seed=1,
                                 dos_method=capi.DOS_FOURIER, window=capi.WINDOW_HANN)
                Dout = np.zeros((S, Ef.size))
                capi.tbpm_sync(ctx)
                t0 = time.perf_counter()
                capi.tbpm_dos(ctx, l2, r, Ef, Dout)
                res[name] = (time.perf_counter() - t0, Dout)
            capi.tbpm_lattice_destroy(l2)
            Ms = capi.tbpm_truncation_order(Nseq * math.pi)
            conc_m = (Ms + (Ms & 1)) // 2
            seq_m = Nseq * (capi.tbpm_truncation_order(math.pi) - 1)
            sweep.append({
                "D_H": i2.coordination + 1, "n_steps": Nseq,
                "wall_s_concurrent": res["concurrent_m"][0], "wall_s_sequential": res["sequential"][0],
                "speedup_wall": res["sequential"][0] / res["concurrent_m"][0],
                "speedup_theory": seq_m / conc_m,
                "site_updates_per_s_concurrent": conc_m * i2.n_sites * S / res["concurrent_m"][0],
                "site_updates_per_s_sequential": seq_m * i2.n_sites * S / res["sequential"][0],
                "max_rel_dos_difference": float(np.max(np.abs(res["concurrent_m"][1] - res["sequential"][1])) /
                                                np.max(np.abs(res["sequential"][1])))})
        out["dh_sweep"] = sweep

    if rank == 0 and args.forms:
        out["forms"] = dense_forms(capi, ctx, desc, S, args.forms_steps)

    if rank == 0 and not args.no_cpu and world == 1:
        try:
            out["cpu_baseline"] = cpu_baseline_obj(work, oracle_sample(work, args.cpu_seconds))
        except Exception as exc:
            out["cpu_baseline"] = {"value": None, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
                                   "sample": f"failed: {exc!r}"[:300]}
    capi.tbpm_destroy(ctx)
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


def main():
    args = parse()
    work = WORKLOADS[args.workload]
    if args.serving:
        run_serving(args)
        return
    if args.impl == "reference":
        run_reference(args, work)
    elif work.lattice.cutoff > 0:
        run_dense(args, work)
    elif work.n_moments == 0:
        run_state_based(args, work)
    else:
        run_gpu(args, work)


if __name__ == "__main__":
    main()
