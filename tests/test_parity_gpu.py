"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Small cases run whole frames (several tiles, ragged right/bottom tiles, image
borders, tiny and maximal windows); the 720p and 1080p workloads run at full
size with the CUDA path in its benchmark launch configuration and the oracle
evaluating a band of rows (it reads the full frames, so windows and borders
are the real ones).
"""
import numpy as np
import pytest

from lockstep import run
from oracle import ADAPTIVE, EXHAUSTIVE, Oracle, OracleConfig
from scenes import Scene, SceneConfig, preset

pytestmark = pytest.mark.gpu


# which regression kernel serves adaptive frames: the library's choice, the
# tile-staged kernel always, or the sparse kernel always, with its window boxes
# staged in shared memory (where they fit) or read through L1 only:
# (sparse threshold, sparse staging); None = the library's default
PATHS = {"auto": (None, None), "staged": ("0", None), "sparse": ("4294967295", None),
         "sparse_l1": ("4294967295", "0")}


def _sim(W, H, r, T, C, mode, rgb, capacity=1 << 22, path="auto"):
    import os
    from paper_2303_02608_gb300 import SimConfig, Simulator
    keys = ("ESIM_AD_SPARSE_MAX", "ESIM_AD_SPARSE_STAGE")
    old = {k: os.environ.pop(k, None) for k in keys}
    for k, v in zip(keys, PATHS[path]):
        if v is not None:
            os.environ[k] = v
    try:
        return Simulator(SimConfig(width=W, height=H, radius=r, frames=T, contrast=C, mode=mode, rgb=rgb,
                                   event_capacity=capacity))
    finally:
        for k in keys:
            os.environ.pop(k, None)
            if old[k] is not None:
                os.environ[k] = old[k]


def _orc(W, H, r, T, C, mode, rgb):
    return Oracle(OracleConfig(W, H, radius=r, frames=T, channels=3 if rgb else 1, mode=mode, contrast=C))


def _case(scene_cfg, r, T, C, mode, n_frames, rows=None, strict=True, path="auto"):
    sc = Scene(scene_cfg)
    frames = sc.sequence(n_frames)
    W, H, rgb = scene_cfg.width, scene_cfg.height, scene_cfg.rgb
    sim = _sim(W, H, r, T, C, mode, rgb, path=path)
    orc = _orc(W, H, r, T, C, mode, rgb)
    rep = run(frames, sim, orc, C, rows=rows, strict=strict, adaptive=(mode == ADAPTIVE))
    sim.close()
    return rep


@pytest.mark.parametrize("mode,path", [(ADAPTIVE, "staged"), (ADAPTIVE, "sparse"), (ADAPTIVE, "sparse_l1"),
                                       (EXHAUSTIVE, "auto")])
@pytest.mark.parametrize("strict", [True, False])
def test_disc_64(mode, path, strict):
    """64x64 disc, 8 frames, 7x7x3 window, C = 0.2, luminance (the tiny workload)."""
    rep = _case(preset("disc64"), 3, 3, 0.2, mode, 8, strict=strict, path=path)
    assert rep["events"] > 0 and rep["regressed"] > 0
    total = 64 * 64 * 8
    assert rep["flag_ambiguous"] + rep["event_ambiguous"] < 0.001 * total + 2


@pytest.mark.parametrize("mode,path", [(ADAPTIVE, "staged"), (ADAPTIVE, "sparse"), (ADAPTIVE, "sparse_l1"),
                                       (EXHAUSTIVE, "auto")])
def test_ragged_rects(mode, path):
    """77x45 RGB rectangles (ragged tiles both ways), 5x5x2 window."""
    cfg = SceneConfig(kind="rects", width=77, height=45, frames=6, spp=4, seed=3, rgb=True,
                      n_rects=8, bg_depth=10.0)
    rep = _case(cfg, 2, 2, 0.15, mode, 6, path=path)
    assert rep["regressed"] > 0


@pytest.mark.parametrize("W,H,r,T", [(1, 1, 1, 1), (5, 3, 1, 2), (33, 9, 1, 1), (40, 70, 15, 4),
                                     (70, 40, 15, 16)])
def test_edge_shapes(W, H, r, T):
    """Single pixel, smaller than a tile, radius 1, the maximum radius (15) and
    temporal window (16), through both adaptive regression kernels."""
    cfg = SceneConfig(kind="rects", width=W, height=H, frames=max(3, min(T + 2, 18)), spp=2, seed=5,
                      rgb=True, n_rects=6, bg_depth=10.0)
    _case(cfg, r, T, 0.15, ADAPTIVE, cfg.frames, path="staged")
    _case(cfg, r, T, 0.15, ADAPTIVE, cfg.frames, path="sparse")
    _case(cfg, r, T, 0.15, EXHAUSTIVE, 3)


def test_static_scene_no_events():
    """Noise-free static input: no pixel is flagged after frame 0 and nothing fires."""
    from paper_2303_02608_gb300 import ESIM_AD_ADAPTIVE
    sc = Scene(preset("disc64", disc_velocity=(0.0, 0.0)))
    c = sc.clean(0)
    fr = {k: c[k].float().contiguous().cuda() for k in ("radiance", "normal", "albedo", "depth")}
    for mode in (ADAPTIVE, EXHAUSTIVE):
        sim = _sim(64, 64, 3, 3, 0.2, mode, False)
        for _ in range(5):
            sim.push(fr)
        _, flags = sim.denoised()
        if mode == ESIM_AD_ADAPTIVE:
            assert int(flags.sum()) == 0
        assert len(sim.events()) == 0
        sim.close()


@pytest.mark.parametrize("mode,rows,path", [(ADAPTIVE, (352, 368), "auto"), (ADAPTIVE, (352, 368), "staged"),
                                            (EXHAUSTIVE, (352, 360), "auto"), (ADAPTIVE, (0, 8), "auto"),
                                            (ADAPTIVE, (712, 720), "staged")])
def test_720p_band(mode, rows, path):
    """The paper-scale workload at full size (1280x720 RGB, 15x15x5, C = 0.15),
    7 frames so the temporal window fills; oracle on a band of rows."""
    rep = _case(preset("rects720p"), 7, 5, 0.15, mode, 7, rows=rows, path=path)
    assert rep["regressed"] > 0


def test_1080p_band():
    """1920x1080, 1 spp-equivalent noise, 15x15x5, C = 0.1 (adaptive); band of rows."""
    rep = _case(preset("rects1080p"), 7, 5, 0.1, ADAPTIVE, 6, rows=(536, 544))
    assert rep["regressed"] > 0


def test_1080p_three_bands_20_frames_free_running():
    """The benchmark's 1080p workload (FP32 form) over 20 frames, free-running:
    the oracle keeps its own models except at threshold-ambiguous pixels;
    bands at the top, middle and bottom of the image."""
    from lockstep import run_bands
    sc = preset("rects1080p")
    frames = Scene(sc).sequence(20)
    bands = [(0, 8), (536, 544), (1072, 1080)]
    sim = _sim(sc.width, sc.height, 7, 5, 0.1, ADAPTIVE, True)
    orcs = [_orc(sc.width, sc.height, 7, 5, 0.1, ADAPTIVE, True) for _ in bands]
    reps = run_bands(frames, sim, orcs, 0.1, bands, strict=False)
    sim.close()
    assert all(r["frames"] == 20 and r["regressed"] > 0 for r in reps)
    assert sum(r["events"] for r in reps) > 0


@pytest.mark.parametrize("path", ["auto", "staged"])
def test_pan1080p_band_paper_density(path):
    """The paper-density workload: rectangles over a textured background seen
    by a panning camera (14-27% of the pixels flagged per frame, where the
    tile-staged kernel serves the flagged-tile queue); two bands."""
    from lockstep import run_bands
    sc = preset("pan1080p")
    frames = Scene(sc).sequence(8)
    bands = [(400, 408), (800, 808)]
    sim = _sim(sc.width, sc.height, 7, 5, 0.1, ADAPTIVE, True, path=path)
    orcs = [_orc(sc.width, sc.height, 7, 5, 0.1, ADAPTIVE, True) for _ in bands]
    reps = run_bands(frames, sim, orcs, 0.1, bands, strict=True)
    phi = sim.stats()["regressions"] / (8 * sc.width * sc.height)
    sim.close()
    assert all(r["frames"] == 8 for r in reps)
    assert phi > 0.1, phi


@pytest.mark.parametrize("mode,path", [(ADAPTIVE, "staged"), (ADAPTIVE, "sparse")])
def test_variance_guard(mode, path):
    """Optional guard (kappa = 3, the frame's variance plane): flags also where
    the log brightness itself moved past C + 3 sigma_y; both sides apply it."""
    import os
    from paper_2303_02608_gb300 import SimConfig, Simulator
    cfg = SceneConfig(kind="rects", width=96, height=72, frames=8, spp=8, seed=21, rgb=True, n_rects=8,
                      bg_depth=10.0)
    frames = Scene(cfg).sequence(8)
    keys = ("ESIM_AD_SPARSE_MAX", "ESIM_AD_SPARSE_STAGE")
    old = {k: os.environ.pop(k, None) for k in keys}
    if PATHS[path][0] is not None:
        os.environ["ESIM_AD_SPARSE_MAX"] = PATHS[path][0]
    try:
        sim = Simulator(SimConfig(width=96, height=72, radius=3, frames=3, contrast=0.15, mode=mode, rgb=True,
                                  guard_kappa=3.0))
    finally:
        for k in keys:
            os.environ.pop(k, None)
            if old[k] is not None:
                os.environ[k] = old[k]
    orc = Oracle(OracleConfig(96, 72, radius=3, frames=3, channels=3, mode=mode, contrast=0.15, guard_kappa=3.0))
    rep = run(frames, sim, orc, 0.15, adaptive=True)
    sim.close()
    plain = _case(cfg, 3, 3, 0.15, mode, 8, path=path)
    # the guard only adds regressions
    assert rep["regressed"] >= plain["regressed"] and rep["events"] > 0
