"""The N > 1 path of bench.py on CPU: two gloo ranks.

bench.py runs one independent replica of the workload per GPU; the job's
step time is the maximum over ranks (every rank waits for the slowest) and
its throughput counts the units of all ranks.  Here two CPU processes form a
gloo process group (127.0.0.1) and run those two reductions with different
rank-local times; the reference arm returns on ranks other than 0.
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t_local = 0.5 + rank          # rank 1 is the slow one
        t = bench.max_over_ranks(t_local, dist)
        v = bench.job_throughput(1000, t, world)
        dist.barrier()
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_step_time_and_count_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in out:
        assert t == 1.5                  # the maximum over ranks, on every rank
        assert v == pytest.approx(2 * 1000 / 1.5)


def test_without_a_process_group_the_local_numbers_stand():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25, None) == 0.25
    assert bench.job_throughput(10, 0.5, 1) == 20.0


def test_reference_arm_does_nothing_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        warmup, steps, gpus = 3, 2, 2
    bench.run_reference(Args(), rank=1, world=2)
    assert capsys.readouterr().out == ""
