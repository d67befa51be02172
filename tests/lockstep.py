"""Lock-step comparison of the CUDA simulator with the FP64 oracle.

Per frame, both sides process the same seeded input.  In ``strict`` mode the
oracle first adopts the GPU's per-pixel model (L_last, beta, x^c), so every
frame checks the transition function itself: the flag decision of
Proposition 1, the regression, and Eq. 1 emission.  In free-running mode the
oracle keeps its own model except at pixels whose decision was ambiguous,
where it adopts the GPU's (the protocol for decisions that sit on a
threshold).

Tolerances (the bar for floating point):
  * alpha (denoised log brightness): |alpha_gpu - alpha_oracle| <= 1e-4;
  * flag decisions exact unless C lies between the GPU's and the oracle's own
    test statistics |beta^T (x^c - xhat^c)| widened by 1e-4;
  * event counts and lists exact unless a crossing k*C (k >= 1) lies between
    the two sides' |Delta L| widened by 1e-4 (Delta L within 1e-4 of p*C).
"""
from __future__ import annotations

import numpy as np

ALPHA_TOL = 1e-4
DECISION_TOL = 1e-4


def counts_from_events(ev, H, W, frame=None):
    m = np.zeros((H, W), np.int64)
    if len(ev) == 0:
        return m
    if isinstance(ev, np.ndarray) and ev.dtype.names:
        f, x, y, p = ev["frame"], ev["x"], ev["y"], ev["polarity"]
    else:
        f, x, y, p = ev[:, 0], ev[:, 1], ev[:, 2], ev[:, 3]
    sel = np.ones(len(f), bool) if frame is None else (f == frame)
    np.add.at(m, (y[sel].astype(np.int64), x[sel].astype(np.int64)), p[sel].astype(np.int64))
    return m


def canonical_ok(ev, W) -> bool:
    if len(ev) < 2:
        return True
    key = ev["frame"].astype(np.int64) * (1 << 32) + ev["y"].astype(np.int64) * W + ev["x"].astype(np.int64)
    return bool(np.all(np.diff(key) >= 0))


def _straddles(a, b, thr, tol):
    """True where the threshold thr lies between |a| and |b| (widened by tol)."""
    lo = np.minimum(np.abs(a), np.abs(b)) - tol
    hi = np.maximum(np.abs(a), np.abs(b)) + tol
    return (lo <= thr) & (thr <= hi)


def _crossing_between(a, b, C, tol):
    """True where some k*C, k >= 1, lies between |a| and |b| (widened by tol)."""
    lo = np.maximum(np.minimum(np.abs(a), np.abs(b)) - tol, 0.0)
    hi = np.maximum(np.abs(a), np.abs(b)) + tol
    return np.floor(lo / C) != np.floor(hi / C)


def new_report():
    return {"frames": 0, "alpha_max_err": 0.0, "regressed": 0, "flag_ambiguous": 0,
            "event_ambiguous": 0, "events": 0, "adopted": 0}


def adopt_gpu_state(orc, g_st):
    """Give the oracle the GPU's per-pixel model (strict lock-step)."""
    n = len(g_st["l_last"])
    beta9 = np.zeros((n, 9))
    beta9[:, 2:] = g_st["beta"]
    orc.set_state(g_st["l_last"].astype(np.float64), beta9, g_st["xc"].astype(np.float64))


def _guard_margin(fr, l_last, kappa, eps=1e-3):
    """|y - L_last| - (C-free part of the guard threshold kappa * sigma_y), FP64,
    from the frame's radiance (RGB or luminance) and variance."""
    rad = np.asarray(fr["radiance"], np.float64)
    Y = rad[0] if rad.shape[0] == 1 else 0.2126 * rad[0] + 0.7152 * rad[1] + 0.0722 * rad[2]
    y = np.log(Y + eps)
    sig = np.sqrt(np.maximum(np.asarray(fr["variance"], np.float64), 0.0)) / (Y + eps)
    return np.abs(y - l_last) - kappa * sig


def compare_frame(t, fr, g_alpha, g_flag, g_ev, g_st, orc, C, band, adaptive, rep, alpha_tol=ALPHA_TOL,
                  strict=True, gpu_state_after=None):
    """Compare one frame after both sides processed it.  g_st is the GPU model
    before the frame (None at t = 0); g_ev holds this frame's GPU events."""
    H, W = band.shape
    n = H * W
    o = orc.outputs()
    o_ev = orc.take_events()
    o_flag = o["flag"].astype(bool)
    amb_f = np.zeros((H, W), bool)
    if adaptive and t > 0:
        # the GPU's own test statistic from its model and this frame's features
        feats = np.concatenate([np.asarray(fr["normal"]), np.asarray(fr["depth"])[None],
                                np.asarray(fr["albedo"])], 0).reshape(7, n).T.astype(np.float64)
        s_g = np.sum(g_st["beta"].astype(np.float64) * (g_st["xc"].astype(np.float64) - feats), 1)
        amb_f = band & _straddles(s_g.reshape(H, W), o["stat"], C, DECISION_TOL)
        kappa = getattr(orc.cfg, "guard_kappa", 0.0)
        if kappa > 0:
            # the guard's decision quantity, from the GPU's level (both sides
            # hold it in strict mode): ambiguous within the tolerance of C
            m = _guard_margin(fr, g_st["l_last"].reshape(H, W).astype(np.float64), kappa)
            amb_f |= band & (np.abs(m - C) <= DECISION_TOL)
    bad_flag = band & ~amb_f & (g_flag != o_flag)
    assert not bad_flag.any(), f"frame {t}: {int(bad_flag.sum())} flag decisions differ " \
                               f"(first at {np.argwhere(bad_flag)[0]})"
    both = band & g_flag & o_flag
    if both.any():
        err = np.abs(g_alpha[both] - o["alpha"][both])
        rep["alpha_max_err"] = max(rep["alpha_max_err"], float(err.max()))
        rep.setdefault("alpha_errors", []).append(err)
        assert err.max() <= alpha_tol, f"frame {t}: alpha error {err.max():.3e} at " \
                                       f"{np.argwhere(both)[int(err.argmax())]}"
    rep["regressed"] += int(both.sum())
    amb_e = np.zeros((H, W), bool)
    if t > 0:
        dl_g = g_alpha - g_st["l_last"].reshape(H, W).astype(np.float64)
        with np.errstate(invalid="ignore"):
            amb_e = both & _crossing_between(dl_g, o["dl"], C, DECISION_TOL)
    amb = amb_f | amb_e
    g_cnt = counts_from_events(g_ev, H, W, frame=t)
    o_cnt = counts_from_events(o_ev, H, W, frame=t)
    if t == 0:
        assert len(g_ev) == 0 and len(o_ev) == 0
    bad_ev = band & ~amb & (g_cnt != o_cnt)
    assert not bad_ev.any(), f"frame {t}: event counts differ at {int(bad_ev.sum())} pixels " \
                             f"(first at {np.argwhere(bad_ev)[0]})"
    assert canonical_ok(g_ev, W), f"frame {t}: events not in canonical order"
    # exact list equality on unambiguous pixels of the band
    if len(g_ev):
        keep_g = band[g_ev["y"], g_ev["x"]] & ~amb[g_ev["y"], g_ev["x"]]
        gl = np.stack([g_ev["frame"][keep_g].astype(np.int64), g_ev["x"][keep_g].astype(np.int64),
                       g_ev["y"][keep_g].astype(np.int64), g_ev["polarity"][keep_g].astype(np.int64)], 1)
    else:
        gl = np.zeros((0, 4), np.int64)
    if len(o_ev):
        keep_o = band[o_ev[:, 2], o_ev[:, 1]] & ~amb[o_ev[:, 2], o_ev[:, 1]]
        ol = o_ev[keep_o].astype(np.int64)
    else:
        ol = np.zeros((0, 4), np.int64)
    assert gl.shape == ol.shape and np.array_equal(gl, ol), f"frame {t}: event lists differ"
    rep["events"] += int(len(ol))
    rep["flag_ambiguous"] += int(amb_f.sum())
    rep["event_ambiguous"] += int(amb_e.sum())
    if not strict and amb.any():
        # ambiguous pixels take the GPU's model so later frames stay comparable
        st = gpu_state_after()
        ost = orc.state()
        idx = np.flatnonzero(amb)
        ost["l_last"][idx] = st["l_last"][idx]
        ost["beta"][idx, 2:] = st["beta"][idx]
        ost["xc"][idx] = st["xc"][idx]
        orc.set_state(ost["l_last"], ost["beta"], ost["xc"])
        rep["adopted"] += int(len(idx))
    rep["frames"] += 1


def run(frames, sim, orc, C, rows=None, strict=True, adaptive=True, report=None, alpha_tol=ALPHA_TOL):
    """Drive both sides over `frames` (dicts of CPU tensors).  Returns a report
    and raises AssertionError on the first out-of-tolerance frame."""
    import torch

    H, W = orc.cfg.height, orc.cfg.width
    r0, r1 = (0, H) if rows is None else rows
    rep = report if report is not None else new_report()
    band = np.zeros((H, W), bool)
    band[r0:r1] = True
    for t, fr in enumerate(frames):
        g_st = sim.get_state() if t > 0 else None
        if t > 0 and strict:
            adopt_gpu_state(orc, g_st)
        if "gpu" in fr:            # inputs in a storage format; fr holds their dequantised values
            gpu_in = {k: v.cuda() for k, v in fr["gpu"].items()}
        else:
            gpu_in = {k: fr[k].cuda() for k in ("radiance", "normal", "albedo", "depth", "variance") if k in fr}
        sim.push(gpu_in)
        orc.push(fr, None if rows is None else rows)
        g_alpha, g_flag = sim.denoised()
        g_alpha = g_alpha.cpu().numpy().astype(np.float64)
        g_flag = g_flag.cpu().numpy().astype(bool)
        g_ev = sim.events()
        torch.cuda.synchronize()
        compare_frame(t, fr, g_alpha, g_flag, g_ev, g_st, orc, C, band, adaptive, rep, alpha_tol, strict,
                      gpu_state_after=sim.get_state)
    return rep


def run_bands(frames, sim, orcs, C, bands, strict=False, adaptive=True, alpha_tol=ALPHA_TOL):
    """As run(), with one oracle per band of rows (bands: list of (r0, r1),
    orcs: one oracle per band); the CUDA path runs once over whole frames and
    every band is compared each frame.  Returns one report per band."""
    import torch

    H, W = orcs[0].cfg.height, orcs[0].cfg.width
    masks = []
    for r0, r1 in bands:
        m = np.zeros((H, W), bool)
        m[r0:r1] = True
        masks.append(m)
    reps = [new_report() for _ in bands]
    for t, fr in enumerate(frames):
        g_st = sim.get_state() if t > 0 else None
        if t > 0 and strict:
            for orc in orcs:
                adopt_gpu_state(orc, g_st)
        if "gpu" in fr:
            gpu_in = {k: v.cuda() for k, v in fr["gpu"].items()}
        else:
            gpu_in = {k: fr[k].cuda() for k in ("radiance", "normal", "albedo", "depth", "variance") if k in fr}
        sim.push(gpu_in)
        for orc, rows in zip(orcs, bands):
            orc.push(fr, rows)
        g_alpha, g_flag = sim.denoised()
        g_alpha = g_alpha.cpu().numpy().astype(np.float64)
        g_flag = g_flag.cpu().numpy().astype(bool)
        g_ev = sim.events()
        torch.cuda.synchronize()
        for orc, band, rep in zip(orcs, masks, reps):
            compare_frame(t, fr, g_alpha, g_flag, g_ev, g_st, orc, C, band, adaptive, rep, alpha_tol, strict,
                          gpu_state_after=sim.get_state)
    return reps

