"""The N > 1 path of bench.py on the host: world_size-2 gloo process groups
(CPU only).  Under torchrun every rank solves its own problem (replicas, no
data-path collective); the job's time is the slowest rank's and the
throughput counts every rank's solves."""
import argparse
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q, steps):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from paper_2110_02485_gb300 import synth
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    own_ms = 100.0 + 40.0 * r                       # rank 1 is the slow one
    dist.barrier()
    ms = bench.max_over_ranks(own_ms, w, "cpu")
    value = bench.job_throughput(w, steps, ms)
    seed = bench.replica_seed(synth.CONFIGS["n32"], r)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, ms, value, seed))


def run_ranks(world, steps=5):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, steps)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_solves():
    out = run_ranks(2)
    slowest = 140.0
    for r, (rank, world, local, ms, value, seed) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert ms == slowest                         # every rank sees the job's time
        sys.path.insert(0, ROOT)
        import bench
        assert value == pytest.approx(2 * bench.SOLVES_PER_STEP * 5 / (slowest / 1e3))
    assert out[0][5] != out[1][5]                    # independent problems per rank


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(1, 4, 1000.0) == pytest.approx(4 * bench.SOLVES_PER_STEP)


def test_reference_arm_other_ranks_exit_without_work(capsys):
    """Under torchrun only rank 0 runs the oracle and prints; rank 1 returns at once."""
    sys.path.insert(0, ROOT)
    import bench
    a = argparse.Namespace(steps=1, warmup=0, config="n32")
    assert bench.run_reference(a, 1, 2) is None
    assert capsys.readouterr().out == ""
