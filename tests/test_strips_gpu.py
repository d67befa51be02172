"""Strip split of one sequence, run on one GPU: the ranks' contexts one after
another, each fed the held rows of every frame (its own rows plus the halo
rows the exchange would deliver), against the whole-frame simulator on the
same frames.

Exhaustive mode regresses every pixel with one lane in a fixed window order,
so an owned pixel's arithmetic does not depend on where its strip starts: the
owned rows' alpha must equal the whole frame's bit for bit, and the merged
event list must equal its list exactly, free-running over the sequence.

Adaptive mode splits a flagged pixel's window over a number of lanes that
depends on its neighbours in the flagged list, so the sums are rounded in
another order.  There the comparison is lock-step: before each frame every
context (the whole-frame one included) takes the whole-frame context's
per-pixel model, so flag decisions must be equal exactly, alpha of the
regressed pixels within 1e-4, and each pixel's events equal unless a crossing
k*C lies between the two sides' Delta L widened by 1e-4.
"""
import numpy as np
import pytest
import torch

from lockstep import _crossing_between, canonical_ok, counts_from_events
from scenes import Scene, SceneConfig

pytestmark = pytest.mark.gpu

ALPHA_TOL = 1e-4
EVENT_TOL = 1e-4
PLANES = ("radiance", "normal", "albedo", "depth")


def _scene(W, H, n, seed):
    cfg = SceneConfig(kind="rects", width=W, height=H, frames=n, spp=2, seed=seed, rgb=True, n_rects=14,
                      bg_depth=10.0)
    return [{k: fr[k].cuda() for k in PLANES} for fr in Scene(cfg).sequence()]


def _contexts(cfg, world):
    from paper_2303_02608_gb300 import Simulator
    from paper_2303_02608_gb300.strips import StripSimulator
    return Simulator(cfg), [StripSimulator(cfg, world, k) for k in range(world)]


@pytest.mark.parametrize("world,W,H,r,T", [(2, 96, 70, 3, 3), (3, 80, 61, 5, 2), (4, 64, 64, 7, 3)])
def test_strips_exhaustive_bitwise(world, W, H, r, T):
    import paper_2303_02608_gb300 as m
    from paper_2303_02608_gb300 import SimConfig
    from paper_2303_02608_gb300.strips import held_frame, merge_events
    cfg = SimConfig(width=W, height=H, radius=r, frames=T, contrast=0.15, mode=m.ESIM_AD_EXHAUSTIVE)
    full, strips = _contexts(cfg, world)
    ev_full, ev_strips = [], [[] for _ in strips]
    for t, fr in enumerate(_scene(W, H, 6, seed=11 + world)):
        full.push(fr)
        for s in strips:
            s.push(held_frame(fr, s.rows))
        a_f, f_f = full.denoised()
        for s in strips:
            a_s, f_s = s.denoised()
            lo, hi = s.rows["lo"], s.rows["hi"]
            assert torch.equal(a_s, a_f[lo:hi]), f"frame {t}: alpha of rows {lo}-{hi} differs"
            assert torch.equal(f_s, f_f[lo:hi])
        ev_full.append(full.events())
        for k, s in enumerate(strips):
            ev_strips[k].append(s.events())
    whole = np.concatenate(ev_full)
    merged = merge_events([np.concatenate(e) for e in ev_strips], [s.rows["lo"] for s in strips])
    assert len(whole) > 100
    assert canonical_ok(merged, W)
    for f in ("frame", "x", "y", "polarity"):
        assert np.array_equal(merged[f], whole[f]), f
    full.close()
    for s in strips:
        s.close()


def _lockstep(cfg, world, frames, to_gpu):
    """Adaptive lock-step of the strips against the whole frame; returns the
    largest alpha difference, the number of regressed pixels compared and of
    events, and the number of pixels excused at a crossing."""
    from paper_2303_02608_gb300.strips import held_frame, merge_events
    W, H, C = cfg.width, cfg.height, cfg.contrast
    full, strips = _contexts(cfg, world)
    worst, n_reg, n_ev, excused = 0.0, 0, 0, 0
    for t, fr in enumerate(frames):
        g = to_gpu(fr)
        if t > 0:
            st = full.get_state()
            full.set_state(st["l_last"], st["beta"], st["xc"])
            for s in strips:
                s.set_state(st["l_last"], st["beta"], st["xc"])
            l_last = st["l_last"].reshape(H, W).astype(np.float64)
        full.push(g)
        for s in strips:
            s.push(held_frame(g, s.rows))
        a_f, f_f = full.denoised()
        a_f, f_f = a_f.cpu().numpy(), f_f.cpu().numpy()
        a_s = np.zeros_like(a_f)
        f_s = np.zeros_like(f_f)
        for s in strips:
            a, f = s.denoised()
            a_s[s.rows["lo"]:s.rows["hi"]] = a.cpu().numpy()
            f_s[s.rows["lo"]:s.rows["hi"]] = f.cpu().numpy()
        assert np.array_equal(f_s, f_f), f"frame {t}: flag decisions differ"
        reg = f_f.astype(bool)
        if reg.any():
            d = np.abs(a_s[reg].astype(np.float64) - a_f[reg])
            worst = max(worst, float(d.max()))
            n_reg += int(reg.sum())
            assert d.max() <= ALPHA_TOL, f"frame {t}: alpha differs by {d.max():.3e}"
        ev_f = full.events()
        ev_s = merge_events([s.events() for s in strips], [s.rows["lo"] for s in strips])
        assert canonical_ok(ev_s, W)
        n_ev += len(ev_f)
        if t == 0:
            assert len(ev_f) == 0 and len(ev_s) == 0
            continue
        c_f = counts_from_events(ev_f, H, W)
        c_s = counts_from_events(ev_s, H, W)
        amb = _crossing_between(a_f - l_last, a_s - l_last, C, EVENT_TOL) & reg
        bad = (c_f != c_s) & ~amb
        assert not bad.any(), f"frame {t}: event counts differ at {np.argwhere(bad)[:5].tolist()}"
        excused += int(((c_f != c_s) & amb).sum())
    full.close()
    for s in strips:
        s.close()
    return worst, n_reg, n_ev, excused


@pytest.mark.parametrize("world,W,H,r,T", [(2, 96, 70, 3, 3), (3, 128, 90, 7, 3)])
def test_strips_adaptive_lockstep(world, W, H, r, T):
    import paper_2303_02608_gb300 as m
    from paper_2303_02608_gb300 import SimConfig
    cfg = SimConfig(width=W, height=H, radius=r, frames=T, contrast=0.15, mode=m.ESIM_AD_ADAPTIVE)
    worst, n_reg, n_ev, excused = _lockstep(cfg, world, _scene(W, H, 6, seed=5 + world), lambda f: f)
    print(f"strips {world}: alpha max difference {worst:.3e} over {n_reg} regressions; "
          f"{n_ev} events, {excused} pixels excused at a crossing")
    assert n_reg > W * H and n_ev > 100 and excused <= max(2, n_reg // 1000)


def test_strips_adaptive_lockstep_precision_form():
    """The headline form: FP16 log brightness and BF16 features, mixed
    precision, three strips of a 160 x 96 frame at r = 7, T = 5."""
    import paper_2303_02608_gb300 as m
    from paper_2303_02608_gb300 import SimConfig
    from test_precision_gpu import FSCALE, storage_frame
    W, H = 160, 96
    cfg = SimConfig(width=W, height=H, radius=7, frames=5, contrast=0.1, mode=m.ESIM_AD_ADAPTIVE,
                    radiance_fmt=m.ESIM_AD_LOGLUMA_F16, feature_fmt=m.ESIM_AD_FEAT_BF16,
                    precision=m.ESIM_AD_MIXED, feature_scale=FSCALE)
    scene = SceneConfig(kind="rects", width=W, height=H, frames=6, spp=1, seed=3, rgb=True, n_rects=16,
                        bg_depth=10.0)
    frames = [storage_frame(f)["gpu"] for f in Scene(scene).sequence()]
    worst, n_reg, n_ev, excused = _lockstep(cfg, 3, frames, lambda f: {k: v.cuda() for k, v in f.items()})
    print(f"precision form, 3 strips: alpha max difference {worst:.3e} over {n_reg} regressions; "
          f"{n_ev} events, {excused} pixels excused at a crossing")
    assert n_reg > W * H and n_ev > 100 and excused <= max(2, n_reg // 1000)
