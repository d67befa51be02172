"""Differentiation form on the GPU: forward alpha against the FP64 oracle, and
the hand-written adjoint's gradients against (a) FP64 central finite
differences of the oracle's loss (h = 1e-4) and (b) autograd through the FP64
dense reference (least squares on the augmented system, and the normal
equations), on a 32x32 crop (radiance and the seven bandwidths)."""
import numpy as np
import pytest
import torch

from oracle import EXHAUSTIVE, Oracle, OracleConfig
from scenes import Scene, SceneConfig, preset
from wlr_reference import log_luminance, mse_loss, wlr_alpha

pytestmark = pytest.mark.gpu

R, T, EPS, RIDGE = 3, 3, 1e-3, 1e-4
B = [0.7, 1.3, 1.0, 2.0, 0.5, 1.0, 1.5]


def _crop(cfg, x0, y0, w, h, n):
    fr = Scene(cfg).sequence(n)
    sl = (slice(y0, y0 + h), slice(x0, x0 + w))
    rad = torch.stack([f["radiance"][(slice(None),) + sl] for f in fr]).contiguous()
    feat = torch.stack([torch.cat([f["normal"], f["depth"][None], f["albedo"]])[(slice(None),) + sl]
                        for f in fr]).contiguous()
    clean = torch.stack([f["clean"][(slice(None),) + sl] for f in fr]).contiguous()
    return rad, feat, clean


def _oracle_alpha(rad, feat, b, rows=None):
    F, C, H, W = rad.shape
    o = Oracle(OracleConfig(W, H, radius=R, frames=T, channels=C, mode=EXHAUSTIVE, bandwidth=list(b),
                            ridge=RIDGE, log_eps=EPS))
    out = []
    for t in range(F):
        o.push({"radiance": rad[t].numpy(), "normal": feat[t, 0:3].numpy(), "depth": feat[t, 3].numpy(),
                "albedo": feat[t, 4:7].numpy()}, rows)
        out.append(o.outputs()["alpha"])
    return np.stack(out)


def _gpu(rad, feat, clean, b):
    from paper_2303_02608_gb300 import wlr
    rd = rad.cuda().requires_grad_(True)
    bd = torch.tensor(b, dtype=torch.float32, device="cuda", requires_grad=True)
    alpha = wlr(rd, feat.cuda(), bd, radius=R, frames=T, log_eps=EPS, ridge=RIDGE)
    loss = ((alpha - log_luminance(clean.cuda(), EPS)) ** 2).mean()
    loss.backward()
    return alpha.detach().cpu(), rd.grad.cpu(), bd.grad.cpu(), float(loss.detach())


RECTS = SceneConfig(kind="rects", width=160, height=120, frames=6, spp=2, seed=4, rgb=True, n_rects=12,
                    bg_depth=10.0)


def test_forward_alpha_matches_oracle():
    rad, feat, clean = _crop(RECTS, 20, 30, 48, 40, 5)
    alpha, _, _, _ = _gpu(rad, feat, clean, B)
    ref = _oracle_alpha(rad, feat, B)
    err = np.abs(alpha.numpy() - ref).max()
    assert err <= 1e-4, err


@pytest.mark.parametrize("solver", ["lstsq", "solve"])
def test_gradients_match_dense_autograd_reference(solver):
    """Against autograd through the FP64 dense regression: least squares on the
    sqrt(w)-weighted augmented system, and the weighted normal equations."""
    rad, feat, clean = _crop(RECTS, 40, 40, 32, 32, 4)
    _, g_rad, g_b, _ = _gpu(rad, feat, clean, B)
    b64 = torch.tensor(B, dtype=torch.float64, requires_grad=True)
    r64 = rad.double().requires_grad_(True)
    mse_loss(wlr_alpha(r64, feat.double(), b64, R, T, eps=EPS, ridge=RIDGE, solver=solver),
             clean.double(), EPS).backward()
    gb_ref = b64.grad.numpy()
    np.testing.assert_allclose(g_b.numpy(), gb_ref, rtol=2e-3, atol=2e-3 * np.abs(gb_ref).max())
    gr_ref = r64.grad.numpy()
    scale = np.abs(gr_ref).max()
    err = np.abs(g_rad.numpy() - gr_ref)
    print(f"radiance gradient vs FP64 {solver}: max abs {err.max():.3e} (scale {scale:.3e}), "
          f"max rel where |g| > 1e-2 scale {np.max(err[np.abs(gr_ref) > 1e-2 * scale] / np.abs(gr_ref[np.abs(gr_ref) > 1e-2 * scale])):.3e}")
    np.testing.assert_allclose(g_rad.numpy(), gr_ref, rtol=1e-4, atol=1e-5 * scale)


def test_gradients_match_oracle_finite_differences():
    rad, feat, clean = _crop(RECTS, 40, 40, 32, 32, 4)
    _, g_rad, g_b, _ = _gpu(rad, feat, clean, B)
    y_clean = log_luminance(clean.double(), EPS).numpy()

    def loss(r, b):
        return float(np.mean((_oracle_alpha(r, feat, b) - y_clean) ** 2))

    hb = 1e-4
    for j in range(7):
        bp, bm = list(B), list(B)
        bp[j] += hb
        bm[j] -= hb
        fd = (loss(rad, bp) - loss(rad, bm)) / (2 * hb)
        assert g_b[j].item() == pytest.approx(fd, rel=2e-3, abs=1e-6)
    # radiance: h = 1e-4; the oracle reads float32, so the step actually taken
    # is the float32 difference of the perturbed and original values (FP64 sums)
    he = 1e-4
    for (t, c, yy, xx) in [(0, 0, 10, 12), (2, 1, 0, 31), (3, 2, 16, 16), (1, 0, 31, 0)]:
        rp, rm = rad.clone(), rad.clone()
        rp[t, c, yy, xx] += he
        rm[t, c, yy, xx] -= he
        step = float(rp[t, c, yy, xx]) - float(rm[t, c, yy, xx])
        fd = (loss(rp, B) - loss(rm, B)) / step
        assert g_rad[t, c, yy, xx].item() == pytest.approx(fd, rel=2e-3, abs=1e-7)


def test_backward_is_deterministic():
    rad, feat, clean = _crop(RECTS, 0, 0, 64, 48, 4)
    a = _gpu(rad, feat, clean, B)
    b = _gpu(rad, feat, clean, B)
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_full_size_sequence_sampled():
    """The differentiation workload at full size: 512x512, 16 frames, 2 spp;
    alpha sampled on a band of rows against the oracle, gradients finite."""
    sc = Scene(preset("rects512"))
    fr = sc.sequence()
    rad = torch.stack([f["radiance"] for f in fr])
    feat = torch.stack([torch.cat([f["normal"], f["depth"][None], f["albedo"]]) for f in fr])
    clean = torch.stack([f["clean"] for f in fr])
    b = [1.0] * 7
    alpha, g_rad, g_b, loss = _gpu(rad, feat, clean, b)
    ref = _oracle_alpha(rad, feat, b, rows=(250, 254))
    err = np.abs(alpha.numpy()[:, 250:254] - ref[:, 250:254]).max()
    assert err <= 1e-4, err
    assert np.isfinite(loss) and torch.isfinite(g_rad).all() and torch.isfinite(g_b).all()
