"""Evaluation kernels against the evaluation oracle: the plain ESIM step
(lock-step, exact except at pixels whose |dL| lies within 2e-5 of a multiple
k >= 1 of C), and P/R/F/chamfer on simulator-produced and random event sets
(counts within tau exact except for events whose oracle distance lies within
1e-6 of tau; chamfer to 1e-5 relative)."""
import numpy as np
import pytest
import torch

from oracle import quality as Q
from scenes import Scene, SceneConfig, preset

pytestmark = pytest.mark.gpu

TAUS = [5e-4, 1e-3, 3e-3, 1e-2, 3e-2, 0.1]


def _esim_gpu(frames, C, key):
    from paper_2303_02608_gb300 import esim_frame
    H, W = frames[0]["depth"].shape
    l_last = torch.empty(H, W, dtype=torch.float32, device="cuda")
    out = []
    for t, f in enumerate(frames):
        counts = torch.empty(H, W, dtype=torch.int32, device="cuda")
        esim_frame(f[key].cuda().contiguous(), l_last, counts, C, init=(t == 0))
        out.append((counts.cpu().numpy(), l_last.cpu().numpy()))
    return out


@pytest.mark.parametrize("key", ["clean", "radiance"])
def test_esim_frame_matches_oracle(key):
    cfg = SceneConfig(kind="rects", width=96, height=72, frames=10, spp=2, seed=11, rgb=True, n_rects=8,
                      bg_depth=10.0)
    frames = Scene(cfg).sequence(10)
    C = 0.15
    gpu = _esim_gpu(frames, C, key)
    level = None
    ambiguous = total = 0
    for t, f in enumerate(frames):
        y = Q.log_brightness(f[key].numpy(), 1e-3)
        c_o, level_new = Q.esim_step(y, level, C)
        c_g, l_g = gpu[t]
        if level is not None:
            dl = np.abs(y - level)
            # within 2e-5 of k C for some k >= 1 (FP32 log brightness and level)
            amb = (dl > C - 2e-5) & (np.abs(dl / C - np.round(dl / C)) * C < 2e-5)
            bad = (c_o != c_g) & ~amb
            assert not bad.any(), (t, int(bad.sum()))
            ambiguous += int(amb.sum())
            total += amb.size
            # lock-step: ambiguous pixels continue from the GPU's level
            level_new = np.where(amb, l_g.astype(np.float64), level_new)
        else:
            assert not c_g.any()
        np.testing.assert_allclose(l_g, level_new, atol=2e-5)
        level = level_new
    # noise-free pixels that return to an earlier value land exactly on a
    # multiple of C (dL = -p n C): genuine ties, hence a few percent here
    print(f"ambiguous pixel-frames: {ambiguous} of {total}")
    assert ambiguous < 0.05 * total


def _compare(gen, ref, taus=TAUS):
    from paper_2303_02608_gb300 import quality
    g = quality(torch.from_numpy(gen.astype(np.int32)).cuda(), torch.from_numpy(ref.astype(np.int32)).cuda(), taus)
    o = Q.quality(gen, ref, taus)
    assert g["n_gen"] == o["n_gen"] and g["n_ref"] == o["n_ref"]
    for k, tau in enumerate(taus):
        for key, d, w, n in (("precision", o["d_gen"], o["w_gen"], o["n_gen"]),
                             ("recall", o["d_ref"], o["w_ref"], o["n_ref"])):
            near = np.abs(d - tau) < 1e-6
            slack = int(w[near].sum())
            assert abs(g[key][k] - o[key][k]) * max(n, 1) <= slack + 1e-9, (key, tau, g[key][k], o[key][k])
    if np.isinf(o["chamfer"]):
        assert np.isinf(g["chamfer"])
    else:
        assert g["chamfer"] == pytest.approx(o["chamfer"], rel=1e-5, abs=1e-12)
    return g, o


def test_quality_on_simulated_sets():
    """Reference: ESIM on the noise-free frames; generated: ESIM on the noisy
    frames and the adaptive simulator's events."""
    from paper_2303_02608_gb300 import SimConfig, Simulator
    cfg = SceneConfig(kind="rects", width=96, height=72, frames=12, spp=2, seed=5, rgb=True, n_rects=8,
                      bg_depth=10.0)
    frames = Scene(cfg).sequence(12)
    C = 0.15
    ref = np.stack([c for c, _ in _esim_gpu(frames, C, "clean")])
    noisy = np.stack([c for c, _ in _esim_gpu(frames, C, "radiance")])
    _compare(noisy, ref)
    sim = Simulator(SimConfig(width=96, height=72, radius=3, frames=3, contrast=C, rgb=True))
    ours = np.zeros_like(ref)
    for f in frames:
        sim.push({k: f[k].cuda() for k in ("radiance", "normal", "albedo", "depth")})
    ev = sim.events()
    sim.close()
    np.add.at(ours, (ev["frame"].astype(np.int64), ev["y"].astype(np.int64), ev["x"].astype(np.int64)),
              ev["polarity"].astype(np.int64))
    g, o = _compare(ours, ref)
    assert g["n_gen"] > 0 and g["n_ref"] > 0


@pytest.mark.parametrize("shape,density", [((6, 9, 13), 0.05), ((1, 5, 7), 0.3), ((9, 1, 17), 0.2),
                                           ((4, 33, 1), 0.2), ((20, 16, 24), 0.002)])
def test_quality_random_sets(shape, density):
    rng = np.random.default_rng(sum(shape))
    gen = rng.integers(-3, 4, size=shape) * (rng.random(shape) < density)
    ref = rng.integers(-3, 4, size=shape) * (rng.random(shape) < density)
    _compare(gen, ref)


def test_quality_degenerate_sets():
    shape = (5, 8, 8)
    z = np.zeros(shape, np.int64)
    one = z.copy()
    one[2, 3, 4] = 1
    g, _ = _compare(one, one)
    assert g["precision"] == [1.0] * len(TAUS) and g["chamfer"] == 0.0
    g, _ = _compare(one, -one)         # polarity never matches: infinite chamfer
    assert np.isinf(g["chamfer"]) and g["precision"][-1] == 0.0
    g, _ = _compare(z, one)            # nothing generated
    assert g["n_gen"] == 0 and g["recall"][-1] == 0.0
