"""The multi-process path of bench.py on CPU: two gloo ranks agree on the slowest rank's time and
on the whole-job rate, and the reference arm runs and prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = [1.5, 2.25][rank]
    slowest = bench.reduce_max(dist, local_seconds)
    rate = bench.whole_job_rate(1000.0, world, slowest)
    dist.barrier()
    with open(f"{out_path}.{rank}", "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_aggregate(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(f"{out}.{r}")) for r in range(2)]
    for r in res:
        assert r["slowest"] == 2.25
        assert r["rate"] == pytest.approx(2 * 1000.0 / 2.25)


def test_single_process_helpers_need_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(None, 3.0) == 3.0
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_state_based_schedule_matches_table_one_counts():
    """bench.py's pass schedule of the time-block form: one pass per generated Chebyshev term
    (Tab. I amxsy, T_0 included) of which all but the last of each block apply H, and one
    accumulator update per (time, term) pair (Tab. I axpy)."""
    import math
    sys.path.insert(0, ROOT)
    import bench
    from oracle import cost, bessel
    for Nt, b in [(100, 1), (100, 7), (2048, 40), (33, 33)]:
        apps, passes, blocks = bench.state_based_schedule(Nt, b, math.pi, bessel.truncation_order)
        c = cost.block_counts(Nt, b, math.pi)
        assert len(passes) == c["amxsy"]
        assert apps == c["amxsy"] - blocks
        assert sum(p[0] for p in passes) == c["axpy"]


def test_byte_models_of_the_two_forms():
    """The state-block crossings behind the bench line's HBM fractions and byte ratio.  Moment form:
    the initial state is written once, the first one-step pass reads phi_0 and writes phi_1, every
    further one-step pass reads two blocks and writes one, and a four-step pass reads two and writes
    two in place of four one-step passes (8 crossings saved each).  Sequential form, per time step:
    each four-term window pass reads two blocks and writes four in place of four one-step passes
    (6 saved each).  Benchmark figures: M = 4096 moments (2048 steps) and N_t = 1254 steps of
    N(pi) = 20 terms give 2,056 and 76,494 crossings."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import bessel
    import math
    for M in (8, 10, 64, 4096, 8192):
        steps = (M + (M & 1)) // 2
        assert bench.concurrent_m_blocks(M, False) == 3 * steps
        assert bench.concurrent_m_blocks(M, True) == 3 * steps - 8 * ((steps - 1) // 4)
    for n_terms in (2, 5, 6, 20, 33):
        plain = bench.sequential_step_blocks(n_terms, False)
        assert plain == 5 + 3 * (n_terms - 2) + n_terms + 6
        windows = max(0, (n_terms - 2) // 4)  # terms 2.. in fours while four more fit below n_terms
        assert bench.sequential_step_blocks(n_terms, True) == plain - 6 * windows
    n_pi = bessel.truncation_order(math.pi)
    assert n_pi == 20
    assert bench.concurrent_m_blocks(4096, True) == 2056
    assert 1254 * bench.sequential_step_blocks(n_pi, True) == 76494
