"""The N > 1 path of bench.py on the CPU, as two gloo ranks.

Every GPU runs an independent replica (its own seeded program; no collective
on the data path), so what multi-rank runs add is host plumbing: the process
group, the barrier around the timed region, the max over ranks of the step
time and the sum of the units all ranks processed.  These tests run that
plumbing with world size 2 over gloo on 127.0.0.1, and check that the
reference arm's non-zero ranks exit at once without work.
"""
import os
import socket
import subprocess
import sys

import multiprocessing as mp

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, step_ms, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    r, w, _ = bench.dist_env()
    bench.init_dist(w, "gloo")
    bench.barrier(w)
    prog, targ = bench.rank_programs(r, 50)
    units = 1000.0 * (r + 1)
    ms, rate = bench.whole_job_rate(units, step_ms[r], w, "cpu")
    bench.barrier(w)
    q.put((r, ms, rate, float(prog.cx[0]), float(targ.cx[0]), prog.n))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_step_time_and_the_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    step_ms = [12.5, 17.25]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, step_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ms, rate, _, _, n in got:
        assert ms == max(step_ms)                       # every rank sees the slowest rank's time
        assert rate == (1000.0 + 2000.0) / (max(step_ms) * 1e-3)
        assert n == 50
    # replicas: the ranks render different programs and targets
    assert got[0][3] != got[1][3] and got[0][4] != got[1][4]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.whole_job_rate(2.0e9, 20.0, 1, "cpu")
    assert ms == 20.0 and rate == 1.0e11
    a, _ = bench.rank_programs(0)
    b, _ = bench.rank_programs(1)
    assert a.n == b.n == 2000 and not np.array_equal(a.cx, b.cx)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="29999")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120,
                       cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
