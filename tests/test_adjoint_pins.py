"""Pins of the FP64 autograd reference (tests/wlr_reference.py): its alpha equals
the oracle's, and its gradients equal central finite differences of the
oracle's loss (FP64 sums, h = 1e-4, the step taken as the float32 difference
of the perturbed inputs the oracle reads)."""
import numpy as np
import pytest
import torch

from oracle import EXHAUSTIVE, Oracle, OracleConfig
from scenes import Scene, SceneConfig
from wlr_reference import log_luminance, mse_loss, wlr_alpha

R, T, EPS, RIDGE = 2, 2, 1e-3, 1e-4
CFG = SceneConfig(kind="rects", width=12, height=10, frames=3, spp=2, seed=9, rgb=True, n_rects=5,
                  bg_depth=10.0)
B = [0.7, 1.3, 1.0, 2.0, 0.5, 1.0, 1.5]


def _inputs():
    sc = Scene(CFG)
    fr = sc.sequence()
    rad = torch.stack([f["radiance"] for f in fr]).double()
    feat = torch.stack([torch.cat([f["normal"], f["depth"][None], f["albedo"]]) for f in fr]).double()
    clean = torch.stack([f["clean"] for f in fr]).double()
    return rad, feat, clean


def _oracle_alpha(rad, feat, b):
    F, C, H, W = rad.shape
    o = Oracle(OracleConfig(W, H, radius=R, frames=T, channels=C, mode=EXHAUSTIVE, bandwidth=list(b),
                            ridge=RIDGE, log_eps=EPS))
    out = []
    for t in range(F):
        o.push({"radiance": rad[t].float().numpy(), "normal": feat[t, 0:3].float().numpy(),
                "depth": feat[t, 3].float().numpy(), "albedo": feat[t, 4:7].float().numpy()})
        out.append(o.outputs()["alpha"])
    return np.stack(out)


def _oracle_loss(rad, feat, clean, b):
    a = _oracle_alpha(rad, feat, b)
    return float(np.mean((a - log_luminance(clean, EPS).numpy()) ** 2))


def test_reference_alpha_equals_oracle():
    rad, feat, _ = _inputs()
    a = wlr_alpha(rad, feat, torch.tensor(B, dtype=torch.float64), R, T, eps=EPS, ridge=RIDGE)
    np.testing.assert_allclose(a.numpy(), _oracle_alpha(rad, feat, B), atol=1e-10)


def test_reference_gradients_equal_oracle_finite_differences():
    rad, feat, clean = _inputs()
    b = torch.tensor(B, dtype=torch.float64, requires_grad=True)
    radv = rad.clone().requires_grad_(True)
    loss = mse_loss(wlr_alpha(radv, feat, b, R, T, eps=EPS, ridge=RIDGE), clean, EPS)
    loss.backward()
    hb = 1e-4
    for j in range(7):
        bp, bm = list(B), list(B)
        bp[j] += hb
        bm[j] -= hb
        fd = (_oracle_loss(rad, feat, clean, bp) - _oracle_loss(rad, feat, clean, bm)) / (2 * hb)
        assert b.grad[j].item() == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # h = 1e-4 on the radiance; the oracle reads float32, so the step taken is
    # the float32 difference of the two perturbed values
    he = 1e-4
    for (t, c, yy, xx) in [(0, 0, 4, 5), (1, 1, 0, 0), (2, 2, 9, 11), (1, 0, 5, 3)]:
        rp, rm = rad.clone(), rad.clone()
        rp[t, c, yy, xx] = float(torch.tensor(float(rad[t, c, yy, xx]) + he, dtype=torch.float32))
        rm[t, c, yy, xx] = float(torch.tensor(float(rad[t, c, yy, xx]) - he, dtype=torch.float32))
        step = float(rp[t, c, yy, xx] - rm[t, c, yy, xx])
        fd = (_oracle_loss(rp, feat, clean, B) - _oracle_loss(rm, feat, clean, B)) / step
        assert radv.grad[t, c, yy, xx].item() == pytest.approx(fd, rel=1e-4, abs=1e-9)


def test_least_squares_reference_equals_normal_equations_and_oracle():
    """The augmented least-squares form of the reference (torch.linalg.lstsq on
    sqrt(w) Z stacked on the ridge rows) gives the oracle's alpha, and its
    autograd gradients equal those through the normal equations."""
    rad, feat, clean = _inputs()
    grads = {}
    for solver in ("solve", "lstsq"):
        b = torch.tensor(B, dtype=torch.float64, requires_grad=True)
        radv = rad.clone().requires_grad_(True)
        a = wlr_alpha(radv, feat, b, R, T, eps=EPS, ridge=RIDGE, solver=solver)
        if solver == "lstsq":
            np.testing.assert_allclose(a.detach().numpy(), _oracle_alpha(rad, feat, B), atol=1e-10)
        mse_loss(a, clean, EPS).backward()
        grads[solver] = (b.grad.numpy(), radv.grad.numpy())
    np.testing.assert_allclose(grads["lstsq"][0], grads["solve"][0], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(grads["lstsq"][1], grads["solve"][1], rtol=1e-8, atol=1e-12)

