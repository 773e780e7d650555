"""Host logic of the multi-rank bench (replicas, no data-path collective) on
CPU: two gloo ranks agree on the slowest rank's time, every rank reads its
rank and world size from the torchrun environment, and the reference arm
runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        info = bench.dist_info()
        slowest = bench.max_over_ranks(10.0 + 3.5 * rank, torch.device("cpu"))
        # rank 1 of the reference arm returns at once, printing nothing
        quiet = bench.run_reference(None, rank, world) is None if rank else True
        q.put((rank, info, slowest, quiet))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [(0, 2, 0), (1, 2, 1)]
    assert all(g[2] == 13.5 for g in got)
    assert all(g[3] for g in got)
