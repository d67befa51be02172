"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.  Each
rank simulates its own sequence (distinct scene per rank), the timings are
reduced to the slowest rank, and the whole-job rate counts every rank's
pixels.  No GPU and no data-path collective are involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from scenes import Scene
        cfg = bench.rank_scene("disc64", rank)
        frame = Scene(cfg).frame(1, "cpu")["radiance"]
        # per-rank timings: rank 1 is slower on the first, rank 0 on the second
        mine = [10.0 + 5.0 * rank, 7.0 - 2.0 * rank]
        slowest = bench.max_over_ranks(mine, dist, "cpu")
        gathered = [torch.zeros_like(frame) for _ in range(world)]
        dist.all_gather(gathered, frame)
        out[rank] = {"slowest": slowest, "seq": cfg.seq, "seed": cfg.seed,
                     "distinct": not torch.equal(gathered[0], gathered[1]),
                     "rate": bench.whole_job_rate(world, cfg.width * cfg.height, 4, slowest[0])}
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0]["slowest"] == res[1]["slowest"] == [15.0, 7.0]
    assert (res[0]["seq"], res[1]["seq"]) == (0, 1) and res[0]["seed"] != res[1]["seed"]
    assert res[0]["distinct"]
    # two ranks x 64x64 pixels x 4 steps in the slowest rank's 15 ms
    assert res[0]["rate"] == pytest.approx(2 * 64 * 64 * 4 / 15e-3)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
    assert bench.whole_job_rate(1, 100, 10, 1000.0) == pytest.approx(1000.0)
