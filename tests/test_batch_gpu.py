"""Batching form against the FP64 oracle: several sequences of uneven
resolution (ragged tiles, a single-tile image), started at different steps and
going idle at different steps, advanced together through the batch API (one
persistent regression launch per step over one queue).  Every sequence is
compared frame by frame with its own oracle, as a single-sequence context is."""
import os

import numpy as np
import pytest
import torch

from lockstep import adopt_gpu_state, compare_frame, new_report
from oracle import ADAPTIVE, EXHAUSTIVE, Oracle, OracleConfig
from scenes import Scene, SceneConfig

pytestmark = pytest.mark.gpu

SHAPES = [(64, 48), (96, 72), (77, 45), (30, 20), (128, 64)]
R, T, C = 3, 3, 0.15


def _scenes(n_frames, shapes=SHAPES, spp=4):
    out = []
    for i, (w, h) in enumerate(shapes):
        cfg = SceneConfig(kind="rects", width=w, height=h, frames=n_frames, spp=spp, seed=100 + i, seq=i,
                          rgb=True, n_rects=8 if w * h < 200000 else 32, bg_depth=10.0)
        out.append(Scene(cfg).sequence(n_frames))
    return out


def _run(mode, pair, tmp_path, strict=True, kappa=0.0, shapes=SHAPES, spans=None, n_steps=9, r=R, t_win=T, c=C,
         bands=None, spp=4):
    """Drive a batch of len(shapes) sequences for n_steps steps, sequence i
    active during steps spans[i]; every active sequence is compared with its
    own oracle each step (on bands[i] = (r0, r1) rows, or the whole image).
    pair = (tile width, lanes per pixel) forces the autotuned pair; None tunes."""
    from paper_2303_02608_gb300 import Batch, SimConfig
    os.environ["ESIM_AD_CACHE"] = str(tmp_path / "autotune.txt")
    if pair:
        os.environ["ESIM_AD_BATCH_TILE"], os.environ["ESIM_AD_BATCH_LANES"] = str(pair[0]), str(pair[1])
    else:
        os.environ.pop("ESIM_AD_BATCH_TILE", None)
        os.environ.pop("ESIM_AD_BATCH_LANES", None)
    seqs = _scenes(n_steps, shapes, spp)
    spans = spans or [(0, 9), (0, 6), (2, 9), (1, 8), (0, 9)]
    bands = bands or [None] * len(shapes)
    cfgs = [SimConfig(width=w, height=h, radius=r, frames=t_win, contrast=c, mode=mode, guard_kappa=kappa)
            for (w, h) in shapes]
    b = Batch(cfgs)
    orcs = [Oracle(OracleConfig(w, h, radius=r, frames=t_win, channels=3, mode=mode, contrast=c, guard_kappa=kappa))
            for (w, h) in shapes]
    keys = ("radiance", "normal", "albedo", "depth") + (("variance",) if kappa > 0 else ())
    reps = [new_report() for _ in shapes]
    tcount = [0] * len(shapes)
    try:
        for step in range(n_steps):
            active = [spans[i][0] <= step < spans[i][1] for i in range(len(shapes))]
            before = {}
            for i, on in enumerate(active):
                if on and tcount[i] > 0:
                    before[i] = b.get_state(i)
                    if strict:
                        adopt_gpu_state(orcs[i], before[i])
            frames = []
            for i, on in enumerate(active):
                fr = seqs[i][tcount[i]] if on else None
                frames.append(None if fr is None else
                              {k: fr[k].cuda() for k in keys})
            b.step(frames)
            ev = b.events()
            for i, on in enumerate(active):
                if not on:
                    continue
                fr = seqs[i][tcount[i]]
                orcs[i].push(fr, bands[i])
                a, f = b.denoised(i)
                w, h = shapes[i]
                band = np.ones((h, w), bool)
                if bands[i] is not None:
                    band[:] = False
                    band[bands[i][0]:bands[i][1]] = True
                g_ev = ev[ev["seq"] == i]
                inputs = {k: fr[k].numpy() for k in ("normal", "albedo", "depth", "radiance", "variance")}
                compare_frame(tcount[i], inputs,
                              a.cpu().numpy().astype(np.float64), f.cpu().numpy().astype(bool), g_ev,
                              before.get(i), orcs[i], c, band, mode == ADAPTIVE, reps[i], strict=strict,
                              gpu_state_after=lambda i=i: b.get_state(i))
                tcount[i] += 1
        stats = b.stats()
    finally:
        b.close()
        os.environ.pop("ESIM_AD_BATCH_TILE", None)
        os.environ.pop("ESIM_AD_BATCH_LANES", None)
    return reps, stats


@pytest.mark.parametrize("pair", [(32, 8), (32, 16), (32, 32), (16, 8), (64, 16)])
def test_batch_adaptive_matches_oracle(pair, tmp_path):
    reps, stats = _run(ADAPTIVE, pair, tmp_path)
    assert stats["lanes"] == pair[1] and stats["tile"] == (pair[0], 256 // pair[0])
    assert sum(r["events"] for r in reps) > 0 and all(r["regressed"] > 0 for r in reps)


def test_batch_exhaustive_matches_oracle(tmp_path):
    reps, _ = _run(EXHAUSTIVE, (32, 16), tmp_path)
    assert all(r["regressed"] > 0 for r in reps)


def test_batch_autotuner_picks_tile_and_lanes_and_caches(tmp_path):
    """Nine adaptive steps after the last sequence start time the nine (tile
    shape, lanes) pairs; the winner is cached as 100 * shape index + lanes."""
    spans = [(0, 14), (0, 14), (2, 14), (1, 14), (0, 14)]
    reps, stats = _run(ADAPTIVE, None, tmp_path, strict=False, spans=spans, n_steps=14)
    assert stats["lanes"] in (8, 16, 32) and stats["tile"] in ((16, 16), (32, 8), (64, 4))
    text = (tmp_path / "autotune.txt").read_text()
    code = 100 * {16: 0, 32: 1, 64: 2}[stats["tile"][0]] + stats["lanes"]
    assert "batch r=3 T=3" in text and text.strip().endswith(str(code))


def test_batch_variance_guard(tmp_path):
    """The optional variance guard in the batched ingest (each sequence's
    variance plane), against per-sequence oracles with the same guard."""
    reps, _ = _run(ADAPTIVE, (32, 8), tmp_path, kappa=3.0)
    assert sum(r["events"] for r in reps) > 0


@pytest.mark.parametrize("pair", [(32, 8), (16, 16)])
def test_batch_benchmark_window_with_1080p_member(pair, tmp_path):
    """The benchmark's window (15x15 x 5 frames, C = 0.15) on mixed
    resolutions with one 1920x1080 member (oracle on a band of rows), the
    members starting and stopping at different steps."""
    shapes = [(1920, 1080), (640, 480), (256, 256), (301, 173)]
    spans = [(0, 7), (1, 7), (0, 5), (2, 7)]
    bands = [(536, 544), (200, 208), None, None]
    reps, stats = _run(ADAPTIVE, pair, tmp_path, shapes=shapes, spans=spans, n_steps=7, r=7, t_win=5, c=0.15,
                       bands=bands, spp=2)
    assert all(r["regressed"] > 0 for r in reps) and sum(r["events"] for r in reps) > 0
