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


def _strip_main(rank, world, port, out, H, W, r):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2303_02608_gb300.strips import halo_exchange, strip_rows
        g = torch.Generator().manual_seed(7)
        frame = torch.rand(8, H, W, generator=g)            # the new frame's ring records, whole image
        s = strip_rows(H, world, rank, r)
        a, b = s["held"]
        local = torch.full((8, b - a, W), float("nan"))
        local[:, s["top"]:s["top"] + s["hi"] - s["lo"]] = frame[:, s["lo"]:s["hi"]]   # own rows only
        halo_exchange(local, H, world, rank, r, dist)
        out[rank] = {"equal": bool(torch.equal(local, frame[:, a:b])), "held": (a, b), "own": (s["lo"], s["hi"])}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,H,r", [(2, 37, 7), (3, 40, 3), (4, 29, 7)])
def test_strip_split_halo_exchange(world, H, r):
    """The strip split's per-frame exchange on gloo ranks: after each rank
    wrote only its owned rows of the new frame, the halo exchange leaves every
    rank holding exactly the whole frame's rows [lo - r, hi + r) (clipped)."""
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_strip_main, args=(k, world, port, out, H, 11, r)) for k in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert all(res[k]["equal"] for k in range(world))
    owns = [res[k]["own"] for k in range(world)]
    assert owns[0][0] == 0 and owns[-1][1] == H and all(owns[k][1] == owns[k + 1][0] for k in range(world - 1))


def test_strip_rows_and_event_merge():
    import numpy as np
    from paper_2303_02608_gb300 import EVENT_DTYPE
    from paper_2303_02608_gb300.strips import merge_events, strip_rows
    with pytest.raises(ValueError):
        strip_rows(9, 2, 0, 7)          # strips thinner than the radius
    s0, s1 = strip_rows(10, 2, 0, 3), strip_rows(10, 2, 1, 3)
    assert (s0["lo"], s0["hi"], s0["top"], s0["bottom"]) == (0, 5, 0, 3)
    assert (s1["lo"], s1["hi"], s1["top"], s1["bottom"]) == (5, 10, 3, 0)
    e0 = np.array([(1, 2, 0, 1), (1, 3, 4, -1), (2, 0, 1, 1)], dtype=EVENT_DTYPE)
    e1 = np.array([(1, 0, 0, 1), (2, 5, 2, -1)], dtype=EVENT_DTYPE)
    m = merge_events([e0, e1], [0, 5])
    key = m["frame"].astype(np.int64) * 1000 + m["y"].astype(np.int64) * 10 + m["x"]
    assert np.all(np.diff(key) > 0) and len(m) == 5 and set(m["y"]) == {0, 4, 1, 5, 7}



class _WindowContext:
    """Stand-in for a simulation context on the CPU: alpha is the mean of
    channel 0 over each pixel's (2r+1)^2 window clipped at the held rows'
    edges (a pixel-local function of its window, as the regression is), and
    a pixel emits one event of polarity sign(alpha - 0.5) when
    |alpha - 0.5| > 0.015."""

    def __init__(self, cfg, stream=None):
        self.cfg = cfg
        self.ev = []
        self.t = 0

    def close(self):
        pass

    def push(self, frame):
        import numpy as np
        from paper_2303_02608_gb300 import EVENT_DTYPE
        x = frame["radiance"][0].numpy().astype(np.float64)
        H, W = x.shape
        assert (H, W) == (self.cfg.height, self.cfg.width)
        r = self.cfg.radius
        a = np.zeros_like(x)
        for y in range(H):
            for c in range(W):
                a[y, c] = x[max(0, y - r):y + r + 1, max(0, c - r):c + r + 1].mean()
        self.alpha = torch.from_numpy(a)
        ys, xs = np.nonzero(np.abs(a - 0.5) > 0.015)
        ev = np.zeros(len(ys), EVENT_DTYPE)
        ev["frame"], ev["x"], ev["y"] = self.t, xs, ys
        ev["polarity"] = np.sign(a[ys, xs] - 0.5)
        self.ev.append(ev)
        self.t += 1

    def events(self):
        import numpy as np
        out = np.concatenate(self.ev)
        self.ev = []
        return out

    def denoised(self):
        return self.alpha, torch.ones_like(self.alpha, dtype=torch.uint8)


@pytest.mark.parametrize("world,H,r", [(2, 37, 3), (3, 40, 5), (4, 29, 7)])
def test_strip_simulators_reproduce_the_whole_frame(world, H, r, monkeypatch):
    """StripSimulator's row bookkeeping on the CPU, with a stand-in context
    whose results are pixel-local functions of clipped windows: the held
    rows cut from each frame, the owned rows kept, and the merged events,
    equal the whole frame's for every split."""
    import numpy as np
    import paper_2303_02608_gb300 as m
    from paper_2303_02608_gb300 import SimConfig
    from paper_2303_02608_gb300.strips import StripSimulator, held_frame, merge_events
    monkeypatch.setattr(m, "Simulator", _WindowContext)
    W = 13
    cfg = SimConfig(width=W, height=H, radius=r)
    full = m.Simulator(cfg)
    strips = [StripSimulator(cfg, world, k) for k in range(world)]
    g = torch.Generator().manual_seed(3)
    for t in range(3):
        fr = {"radiance": torch.rand(3, H, W, generator=g), "depth": torch.rand(H, W, generator=g)}
        full.push(fr)
        for s in strips:
            s.push(held_frame(fr, s.rows))
        a_f, _ = full.denoised()
        for s in strips:
            a_s, f_s = s.denoised()
            assert torch.equal(a_s, a_f[s.rows["lo"]:s.rows["hi"]])
    whole = full.events()
    merged = merge_events([s.events() for s in strips], [s.rows["lo"] for s in strips])
    assert len(whole) > 0
    for f in ("frame", "x", "y", "polarity"):
        assert np.array_equal(merged[f], whole[f]), f
