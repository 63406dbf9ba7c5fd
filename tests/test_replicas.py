"""The bench's multi-GPU mode is replicas only: each rank runs the whole
workload, the ranks meet at barriers and the job time is the slowest rank's.
Checked here with world size 2 over gloo on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ranks = bench.Ranks(dist, torch.device("cpu"))
    ranks.barrier()
    local_ms = 100.0 + 50.0 * rank           # rank 1 is the slower replica
    ms_max = ranks.max(local_ms)
    value = bench.whole_job_rate(512 ** 3, 300, world, ms_max)
    w, r, lr = bench.dist_env()
    out.put((rank, ms_max, value, w, r, lr))
    ranks.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, w, r, lr in res:
        assert ms_max == 150.0
        assert value == pytest.approx(512 ** 3 * 300 * 2 / 0.150)
        assert (w, r, lr) == (2, rank, rank)


def test_single_process_needs_no_collective():
    import bench
    ranks = bench.Ranks(None, torch.device("cpu"))
    ranks.barrier()
    assert ranks.max(3.5) == 3.5
    assert bench.whole_job_rate(100, 10, 1, 1000.0) == pytest.approx(1000.0)

