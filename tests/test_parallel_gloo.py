"""The multi-rank host logic on CPU with gloo, world size 2: view sharding
keeps ray ids disjoint and complete, the benchmark's per-rank views do not
share ray ids, and the timing reduction takes the maximum over ranks."""
import os
import socket

import pytest

import scenes

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2504_06598_gb300 import parallel
    cams = scenes.wavefront_views(7, seed=3, res_range=((16, 16), (64, 48)))
    mine = parallel.shard_views(cams, rank, world)
    ranges = [(c.ray_id_offset, c.ray_id_offset + c.width * c.height) for c in mine]
    gathered = [None] * world
    dist.all_gather_object(gathered, ranges)
    bench_cam = parallel.rank_view(scenes.default_camera(32, 16), rank)
    bench = [None] * world
    dist.all_gather_object(bench, (bench_cam.ray_id_offset, bench_cam.ray_id_offset + 512))
    mx = parallel.max_over_ranks([1.0 + rank, 10.0 - rank])
    if rank == 0:
        out.put((gathered, bench, mx, [(c.ray_id_offset, c.ray_id_offset + c.width * c.height)
                                       for c in cams]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharding_and_reduction_world2():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, bench, mx, all_ranges = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(r for ranks in gathered for r in ranks)
    assert flat == sorted(all_ranges)  # every view exactly once
    for (a0, a1), (b0, b1) in zip(flat, flat[1:]):
        assert a1 <= b0  # disjoint ray ids
    (a0, a1), (b0, b1) = bench
    assert a1 <= b0 or b1 <= a0
    assert mx == [2.0, 10.0]
