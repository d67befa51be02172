"""Second-order regression kernel against its FP64 oracle (oracle/wlr2.py):
every pixel of small rendered-like sequences (ragged rows, clipped windows,
each slot split G = 1, 2, 4, 8, luminance and RGB input, non-unit bandwidths),
sampled centres at 512 x 512 in the launch configuration the benchmark times,
an image smaller than the window, and the closed-form centre weights on a
feature-flat input.  Tolerance: alpha within 1e-4 of the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import wlr2 as O
from scenes import Scene, SceneConfig

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _inputs(W, H, F, rgb=True, seed=3, spp=2):
    cfg = SceneConfig(kind="rects", width=W, height=H, frames=F, spp=spp, seed=seed, rgb=rgb,
                      n_rects=max(4, (W * H) // 150), bg_depth=10.0)
    fr = Scene(cfg).sequence(F)
    rad = torch.stack([f["radiance"] for f in fr]).contiguous()
    feat = torch.stack([torch.cat([f["normal"], f["depth"][None], f["albedo"]]) for f in fr]).contiguous()
    return rad, feat


def _gpu(rad, feat, b=None, **kw):
    from paper_2303_02608_gb300 import wlr2
    bw = None if b is None else torch.tensor(b, dtype=torch.float32, device="cuda")
    return wlr2(rad.cuda(), feat.cuda(), bw, **kw).cpu().double().numpy()


@pytest.mark.parametrize("W,H,F,r,T,rgb,b,groups", [
    (45, 37, 4, 3, 3, True, None, None),
    (40, 29, 3, 2, 1, False, None, None),
    (33, 26, 3, 3, 3, True, (0.6, 1.4, 0.9, 2.5, 0.7, 1.1, 0.8), "2"),
    (33, 26, 3, 3, 3, True, None, "4"),
    (33, 26, 3, 3, 3, True, None, "8"),
    (30, 24, 3, 7, 3, True, None, None),
])
def test_wlr2_matches_oracle(W, H, F, r, T, rgb, b, groups, monkeypatch):
    if groups is not None:
        monkeypatch.setenv("ESIM_AD_WLR2_GROUPS", groups)
    rad, feat = _inputs(W, H, F, rgb)
    g = _gpu(rad, feat, b, radius=r, frames=T)
    o = O.wlr2(rad.numpy(), feat.numpy(), bandwidth=b or (1.0,) * 7, radius=r, frames=T)
    err = np.abs(g - o)
    print(f"{W}x{H}x{F} r={r} T={T} G={groups or 'auto'}: max {err.max():.2e} mean {err.mean():.2e}")
    assert err.max() <= TOL


def test_wlr2_image_smaller_than_window():
    rad, feat = _inputs(5, 3, 2, True, seed=7)
    g = _gpu(rad, feat, radius=3, frames=2)
    o = O.wlr2(rad.numpy(), feat.numpy(), radius=3, frames=2)
    assert np.abs(g - o).max() <= TOL


def test_wlr2_flat_features_closed_form():
    """Constant features leave the coordinate terms only: the centre value is
    the Gaussian-weighted Savitzky-Golay combination of the window."""
    r, F, H, W = 3, 2, 20, 24
    rng = np.random.default_rng(5)
    rad = torch.tensor(rng.uniform(0.1, 3.0, size=(F, 1, H, W)), dtype=torch.float32)
    feat = torch.zeros(F, 7, H, W)
    feat[:, 2], feat[:, 3], feat[:, 4:] = 1.0, 2.0, 0.5
    g = _gpu(rad, feat, radius=r, frames=1, ridge=1e-6)
    y = O.log_brightness(rad.numpy(), 1e-3)
    x = np.arange(-r, r + 1) / r
    gw = np.exp(-0.5 * x ** 2)
    G0, G2, G4 = gw.sum(), (gw * x ** 2).sum(), (gw * x ** 4).sum()
    a = gw * (G4 - G2 * x ** 2) / (G0 * G4 - G2 ** 2)
    c = np.outer(gw / G0, a) + np.outer(a, gw / G0) - np.outer(gw / G0, gw / G0)
    for cy in range(r, H - r):
        for cx in range(r, W - r):
            ref = float((c * y[1, cy - r:cy + r + 1, cx - r:cx + r + 1]).sum())
            assert g[1, cy, cx] == pytest.approx(ref, abs=2e-5)


def test_wlr2_full_size_sampled():
    """512 x 512 x 3 frames, r = 3, T = 3 (the benchmark's kernel and launch
    shape): 400 sampled centres, corners and edges included."""
    W = H = 512
    rad, feat = _inputs(W, H, 3, True, seed=0)
    g = _gpu(rad, feat, radius=3, frames=3)
    rng = np.random.default_rng(1)
    pts = [(t, y, x) for t in (0, 2) for y, x in ((0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (1, 257), (300, 2))]
    pts += [(int(rng.integers(0, 3)), int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(388)]
    o = O.wlr2(rad.numpy(), feat.numpy(), radius=3, frames=3, centres=pts)
    got = np.array([g[t, y, x] for t, y, x in pts])
    assert np.abs(got - o).max() <= TOL


def test_wlr2_deterministic_and_validates():
    from paper_2303_02608_gb300 import EsimError, wlr2
    rad, feat = _inputs(40, 24, 3, True, seed=2)
    a = _gpu(rad, feat, radius=3, frames=3)
    b = _gpu(rad, feat, radius=3, frames=3)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    with pytest.raises((EsimError, ValueError)):
        wlr2(rad.cuda(), feat.cuda(), radius=0)
    with pytest.raises((EsimError, ValueError)):
        wlr2(rad.cuda(), feat.cuda(), radius=3, frames=17)
