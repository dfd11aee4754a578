"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.  Images shard by
rank with no overlap, the step time is the max over ranks, and whole-job throughput
counts every rank's pixels.  (The path itself has no collective: images are
independent.)"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        imgs = list(bench.rank_images(rank, 5))
        local_ms = 10.0 + 7.0 * rank                      # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, imgs)
        # the seeded images of a rank are the same wherever they are drawn
        first = bench._gen((bench.BASE_SEED, imgs[0], 16, 24))
        q.put((rank, imgs, ms, gathered, first.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, i0, ms0, g0, f0), (r1, i1, ms1, g1, f1) = out
    assert set(i0).isdisjoint(i1) and sorted(i0 + i1) == list(range(10))
    assert ms0 == ms1 == 17.0
    assert g0 == g1 == [i0, i1]
    assert f0 == bench._gen((bench.BASE_SEED, i0[0], 16, 24)).tobytes()
    assert bench.job_throughput(1_000_000, world, 4, ms0) == pytest.approx(2 * 4 * 1e6 / 0.017 / 1e6)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert list(bench.rank_images(0, 3)) == [0, 1, 2]
