"""The N > 1 bench path on CPU: world_size-2 gloo ranks run independent
replicas; the barrier and the max-over-ranks timing reduction are the only
collectives, and the reported throughput counts the units of every rank
over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    # CPU ranks even where a GPU is present (init_dist takes NCCL on GPUs)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    import bench
    r, w, local = bench.dist_env()
    tdist = bench.init_dist(w, local)
    assert tdist.get_backend() == "gloo"
    bench.barrier(tdist)
    mine = 1.0 + rank  # rank 1 is slower
    t = bench.max_over_ranks(tdist, mine)
    q.put((rank, t, bench.aggregate_gbs(1536, 1000, w, t)))
    tdist.destroy_process_group()


def test_two_rank_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    assert all(t == 2.0 for _, t, _ in res)
    assert all(abs(g - 1536 * 1000 * 2 / 2.0 / 1e9) < 1e-12 for _, _, g in res)
