"""The benchmark's multi-rank host logic on CPU.  Multi-GPU runs are replicas: each rank tracks its own
sessions with no data-path collective, and the ranks meet only to time the job, which takes as long as its
slowest rank.  Two gloo ranks (spawned processes, rendezvous on 127.0.0.1) check that reduction and the
whole-job rate built on it."""
import multiprocessing as mp
import os
import socket
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, seconds, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = b.max_over_ranks(seconds[rank], world, device="cpu")
        q.put((rank, slowest, b.whole_job_rate(world, 10, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seconds = [1.5, 2.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    # both ranks see the slower rank's 2.5 s; 2 ranks x 10 frames in 2.5 s = 8 frames/s for the job
    assert got == [(0, 2.5, 8.0), (1, 2.5, 8.0)]


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_rate(1, 60, 0.5) == 120.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    # a rank other than 0 returns at once: no oracle work and no output line
    args = types.SimpleNamespace(warmup=3, steps=5, gpus=2)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
