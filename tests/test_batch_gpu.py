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


def _scenes(n_frames):
    out = []
    for i, (w, h) in enumerate(SHAPES):
        cfg = SceneConfig(kind="rects", width=w, height=h, frames=n_frames, spp=4, seed=100 + i, seq=i,
                          rgb=True, n_rects=8, bg_depth=10.0)
        out.append(Scene(cfg).sequence(n_frames))
    return out


def _run(mode, lanes, tmp_path, strict=True, kappa=0.0):
    import paper_2303_02608_gb300 as m
    from paper_2303_02608_gb300 import Batch, SimConfig
    os.environ["ESIM_AD_CACHE"] = str(tmp_path / "autotune.txt")
    if lanes:
        os.environ["ESIM_AD_BATCH_LANES"] = str(lanes)
    else:
        os.environ.pop("ESIM_AD_BATCH_LANES", None)
    n_steps = 9
    seqs = _scenes(n_steps)
    # sequence i runs during steps [start_i, stop_i)
    spans = [(0, 9), (0, 6), (2, 9), (1, 8), (0, 9)]
    cfgs = [SimConfig(width=w, height=h, radius=R, frames=T, contrast=C, mode=mode, guard_kappa=kappa)
            for (w, h) in SHAPES]
    b = Batch(cfgs)
    orcs = [Oracle(OracleConfig(w, h, radius=R, frames=T, channels=3, mode=mode, contrast=C, guard_kappa=kappa))
            for (w, h) in SHAPES]
    keys = ("radiance", "normal", "albedo", "depth") + (("variance",) if kappa > 0 else ())
    reps = [new_report() for _ in SHAPES]
    tcount = [0] * len(SHAPES)
    try:
        for step in range(n_steps):
            active = [spans[i][0] <= step < spans[i][1] for i in range(len(SHAPES))]
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
                orcs[i].push(fr)
                a, f = b.denoised(i)
                w, h = SHAPES[i]
                band = np.ones((h, w), bool)
                g_ev = ev[ev["seq"] == i]
                inputs = {k: fr[k].numpy() for k in ("normal", "albedo", "depth", "radiance", "variance")}
                compare_frame(tcount[i], inputs,
                              a.cpu().numpy().astype(np.float64), f.cpu().numpy().astype(bool), g_ev,
                              before.get(i), orcs[i], C, band, mode == ADAPTIVE, reps[i], strict=strict,
                              gpu_state_after=lambda i=i: b.get_state(i))
                tcount[i] += 1
        stats = b.stats()
    finally:
        b.close()
        os.environ.pop("ESIM_AD_BATCH_LANES", None)
    return reps, stats


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_batch_adaptive_matches_oracle(lanes, tmp_path):
    reps, stats = _run(ADAPTIVE, lanes, tmp_path)
    assert stats["lanes"] == lanes
    assert sum(r["events"] for r in reps) > 0 and all(r["regressed"] > 0 for r in reps)


def test_batch_exhaustive_matches_oracle(tmp_path):
    reps, _ = _run(EXHAUSTIVE, 16, tmp_path)
    assert all(r["regressed"] > 0 for r in reps)


def test_batch_autotuner_picks_and_caches(tmp_path):
    reps, stats = _run(ADAPTIVE, None, tmp_path, strict=False)
    assert stats["lanes"] in (8, 16, 32)
    text = (tmp_path / "autotune.txt").read_text()
    assert "batch r=3 T=3" in text and text.strip().endswith(str(stats["lanes"]))


def test_batch_variance_guard(tmp_path):
    """The optional variance guard in the batched ingest (each sequence's
    variance plane), against per-sequence oracles with the same guard."""
    reps, _ = _run(ADAPTIVE, 8, tmp_path, kappa=3.0)
    assert sum(r["events"] for r in reps) > 0

