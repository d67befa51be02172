"""Bandwidth selection (fitted b_j fed back into the simulator): the fit runs
the library's dense regression and adjoint; the improvement it finds is
confirmed independently by the FP64 oracle's loss at the fitted bandwidths."""
import numpy as np
import pytest
import torch

from oracle import EXHAUSTIVE, Oracle, OracleConfig
from scenes import Scene, SceneConfig

pytestmark = pytest.mark.gpu

R, T, EPS, RIDGE = 3, 3, 1e-3, 1e-4
CFG = SceneConfig(kind="rects", width=160, height=120, frames=6, spp=2, seed=4, rgb=True, n_rects=12, bg_depth=10.0)


def _crop(x0, y0, w, h, n):
    fr = Scene(CFG).sequence(n)
    sl = (slice(y0, y0 + h), slice(x0, x0 + w))
    rad = torch.stack([f["radiance"][(slice(None),) + sl] for f in fr]).contiguous()
    feat = torch.stack([torch.cat([f["normal"], f["depth"][None], f["albedo"]])[(slice(None),) + sl]
                        for f in fr]).contiguous()
    clean = torch.stack([f["clean"][(slice(None),) + sl] for f in fr]).contiguous()
    return rad, feat, clean


def _oracle_loss(rad, feat, clean, b):
    F, C, H, W = rad.shape
    o = Oracle(OracleConfig(W, H, radius=R, frames=T, channels=C, mode=EXHAUSTIVE, bandwidth=list(b),
                            ridge=RIDGE, log_eps=EPS))
    cl = clean.double().numpy()
    Y = 0.2126 * cl[:, 0] + 0.7152 * cl[:, 1] + 0.0722 * cl[:, 2]
    target = np.log(Y + EPS)
    err = []
    for t in range(F):
        o.push({"radiance": rad[t].numpy(), "normal": feat[t, 0:3].numpy(), "depth": feat[t, 3].numpy(),
                "albedo": feat[t, 4:7].numpy()})
        err.append((o.outputs()["alpha"] - target[t]) ** 2)
    return float(np.mean(err))


def test_fitted_bandwidths_lower_the_loss():
    from paper_2303_02608_gb300 import wlr
    from paper_2303_02608_gb300.bandwidth import fit_bandwidths, log_luminance
    rad, feat, clean = _crop(30, 30, 48, 40, 5)
    b, hist = fit_bandwidths(rad.cuda(), feat.cuda(), clean.cuda(), radius=R, frames=T, steps=40, lr=0.2,
                             log_eps=EPS, ridge=RIDGE)
    assert all(np.isfinite(b)) and all(v > 0 for v in b)
    target = log_luminance(clean.cuda(), EPS)

    def gpu_loss(bw):
        a = wlr(rad.cuda(), feat.cuda(), torch.tensor(bw, device="cuda"), radius=R, frames=T, log_eps=EPS,
                ridge=RIDGE)
        return float(((a - target) ** 2).mean())

    l1, lb = gpu_loss([1.0] * 7), gpu_loss(b)
    assert lb < l1 and hist[0] == pytest.approx(l1, rel=1e-5)
    o1, ob = _oracle_loss(rad, feat, clean, [1.0] * 7), _oracle_loss(rad, feat, clean, b)
    print(f"loss b=1: gpu {l1:.6e} oracle {o1:.6e}; fitted b={np.round(b, 3).tolist()}: gpu {lb:.6e} oracle {ob:.6e}")
    assert ob < o1
    assert lb == pytest.approx(ob, rel=1e-3) and l1 == pytest.approx(o1, rel=1e-3)


def test_simulator_accepts_fitted_bandwidths():
    """The fitted b drives the adaptive simulator like any bandwidth vector
    (parity against the oracle with the same b)."""
    from lockstep import run
    from paper_2303_02608_gb300 import SimConfig, Simulator
    b = [0.6, 1.4, 0.9, 2.5, 0.7, 1.1, 0.8]
    frames = Scene(CFG).sequence(5)
    sim = Simulator(SimConfig(width=160, height=120, radius=R, frames=T, contrast=0.15, rgb=True, bandwidth=b))
    orc = Oracle(OracleConfig(160, 120, radius=R, frames=T, channels=3, contrast=0.15, bandwidth=b))
    rep = run(frames, sim, orc, 0.15)
    sim.close()
    assert rep["regressed"] > 0
