"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each checks a closed form, an
exact invariant, a library least-squares solve, or hand-derived event counts,
chosen so that a plausible slip (a dropped term, a flipped sign or offset, a
swapped feature, a wrong window or bandwidth) fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import ADAPTIVE, EXHAUSTIVE, Oracle, OracleConfig


def frame(y_or_rad, normal, albedo, depth):
    rad = np.asarray(y_or_rad, np.float32)
    if rad.ndim == 2:
        rad = rad[None]
    return {"radiance": rad, "normal": np.asarray(normal, np.float32),
            "albedo": np.asarray(albedo, np.float32), "depth": np.asarray(depth, np.float32)}


def uniform_features(H, W, n=(0.0, 0.0, 1.0), a=(0.5, 0.5, 0.5), d=3.0):
    normal = np.stack([np.full((H, W), v) for v in n])
    albedo = np.stack([np.full((H, W), v) for v in a])
    depth = np.full((H, W), d)
    return normal, albedo, depth


def gauss_sum(r, h=1.0, lo=None, hi=None, unit=None):
    unit = r if unit is None else unit
    lo = -r if lo is None else lo
    hi = r if hi is None else hi
    return sum(math.exp(-0.5 * (k / unit / h) ** 2) for k in range(lo, hi + 1))


# ---------------------------------------------------------------- weights (Eq. 5)

@pytest.mark.parametrize("r,T,t", [(1, 1, 0), (3, 3, 2), (3, 3, 1), (2, 4, 5)])
def test_weight_sum_uniform_features(r, T, t):
    """Uniform features: w depends on the coordinate only and factorises, so
    W = T_eff * (sum_k exp(-(k/r)^2/2))^2 at an interior pixel (Eq. 5, h=b=1)."""
    H = W = 2 * r + 5
    o = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=0, mode=EXHAUSTIVE))
    n, a, d = uniform_features(H, W)
    for _ in range(t + 1):
        o.push(frame(np.zeros((H, W)), n, a, d))
    _, _, Wsum = o.wlr_at(W // 2, H // 2)
    T_eff = min(T, t + 1)
    assert Wsum == pytest.approx(T_eff * gauss_sum(r) ** 2, rel=1e-13)
    # corner pixel: the window is clipped to the image, not padded
    _, _, Wc = o.wlr_at(0, 0)
    assert Wc == pytest.approx(T_eff * gauss_sum(r, lo=0) ** 2, rel=1e-13)


@pytest.mark.parametrize("h,b_depth,delta", [(1.0, 1.0, 0.75), (1.0, 2.0, 0.75), (0.5, 1.0, 0.25)])
def test_weight_sum_depth_step(h, b_depth, delta):
    """Depth larger by delta right of the centre column: those neighbours get an
    extra factor exp(-(delta/(h b_depth))^2/2); coordinates use h too."""
    r, H, W = 2, 9, 9
    bw = [1.0] * 7
    bw[3] = b_depth
    o = Oracle(OracleConfig(W, H, radius=r, frames=1, channels=0, mode=EXHAUSTIVE, h=h, bandwidth=bw))
    n, a, d = uniform_features(H, W)
    d = d.copy()
    d[:, W // 2 + 1:] += delta
    o.push(frame(np.zeros((H, W)), n, a, d))
    _, _, Wsum = o.wlr_at(W // 2, H // 2)
    f = math.exp(-0.5 * (delta / (h * b_depth)) ** 2)
    sx = gauss_sum(r, h, lo=-r, hi=0) + f * gauss_sum(r, h, lo=1, hi=r)
    assert Wsum == pytest.approx(gauss_sum(r, h) * sx, rel=1e-13)


def test_weight_sum_pixel_units():
    r, H, W = 2, 7, 7
    o = Oracle(OracleConfig(W, H, radius=r, frames=1, channels=0, mode=EXHAUSTIVE, pixel_units=True))
    n, a, d = uniform_features(H, W)
    o.push(frame(np.zeros((H, W)), n, a, d))
    _, _, Wsum = o.wlr_at(3, 3)
    assert Wsum == pytest.approx(gauss_sum(r, unit=1) ** 2, rel=1e-13)


# ---------------------------------------------------------------- regression (Eqs. 3-4)

def _random_features(rng, H, W):
    normal = rng.uniform(-0.5, 0.5, (3, H, W))
    albedo = rng.uniform(0.2, 0.8, (3, H, W))
    depth = rng.uniform(2.0, 3.0, (H, W))
    return normal, albedo, depth


def _feat_stack(normal, albedo, depth):
    # feature order of the regressors: normal (3), depth (1), albedo (3)
    return np.concatenate([normal, depth[None], albedo], 0).astype(np.float32).astype(np.float64)


def test_linear_field_reproduced_exactly():
    """y = a + g^T x is reproduced: alpha = a + g^T x^c and beta = g (coordinate
    slopes scaled by r because the coordinate regressor is (q - c)/r)."""
    rng = np.random.default_rng(1)
    r, T, H, W = 2, 2, 8, 9
    g = np.array([0.03, -0.02, 0.4, -0.7, 0.25, 1.3, -0.5, 0.9, 0.2])  # dx, dy, n0..2, depth, a0..2
    a0 = 0.3
    o = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=0, mode=EXHAUSTIVE, ridge=1e-12))
    qy, qx = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(T):
        n, a, d = _random_features(rng, H, W)
        f = _feat_stack(n, a, d)
        y = a0 + g[0] * qx + g[1] * qy + np.tensordot(g[2:], f, 1)
        o.push(frame(y, n, a, d))
    for cx, cy in [(4, 4), (0, 0), (8, 7), (2, 5)]:
        theta, R, _ = o.wlr_at(cx, cy)
        exp_alpha = a0 + g[0] * cx + g[1] * cy + g[2:] @ f[:, cy, cx]
        # y was rounded to float32 on input: the fit is exact up to that rounding
        assert theta[0] == pytest.approx(exp_alpha, abs=2e-6)
        np.testing.assert_allclose(theta[1:3], g[:2] * r, atol=2e-5)
        np.testing.assert_allclose(theta[3:], g[2:], atol=5e-5)


def test_model_replaced_at_events_and_kept_otherwise():
    """Fig. 1: the model (beta, x^c) is kept from a pixel's last event.  With
    feature-linear fields (reproduced exactly), frame 1 raises every pixel's
    alpha by more than C: each pixel emits, and its model becomes frame 1's
    fit (beta = g1, x^c = the frame-1 features).  Frame 2 changes one slope
    and one feature slightly (|Delta L| < C): no event, and the model stays
    frame 1's although frame 2 was regressed too (exhaustive mode)."""
    rng = np.random.default_rng(11)
    r, H, W, C = 3, 8, 9, 0.2
    o = Oracle(OracleConfig(W, H, radius=r, frames=1, channels=0, mode=EXHAUSTIVE, contrast=C, ridge=1e-12))
    g0 = rng.uniform(-0.05, 0.05, 7)
    g1 = rng.uniform(-0.05, 0.05, 7)
    g2 = g1 - 0.001 * np.eye(7)[3]                       # depth slope moved
    n0, a0, d0 = _random_features(rng, H, W)
    n1, a1, d1 = _random_features(rng, H, W)
    F0, F1 = _feat_stack(n0, a0, d0), _feat_stack(n1, a1, d1)
    a2 = a1.copy()
    a2[0] += 0.01                                        # albedo red moved
    F2 = _feat_stack(n1, a2, d1)
    o.push(frame(0.1 + np.tensordot(g0, F0, 1), n0, a0, d0))
    alpha0 = o.outputs()["alpha"]
    o.push(frame(1.1 + np.tensordot(g1, F1, 1), n1, a1, d1))
    out1 = o.outputs()
    assert np.all(out1["nev"] >= 1)
    st = o.state()
    np.testing.assert_allclose(st["beta"][:, :2], 0.0, atol=5e-5)
    np.testing.assert_allclose(st["beta"][:, 2:], np.tile(g1, (H * W, 1)), atol=5e-5)
    np.testing.assert_array_equal(st["xc"], F1.reshape(7, -1).T)
    np.testing.assert_allclose(st["l_last"], (alpha0 + out1["nev"] * C).ravel(), atol=1e-12)
    o.push(frame(1.1 + np.tensordot(g2, F2, 1), n1, a2, d1))
    out2 = o.outputs()
    assert np.all(out2["flag"] == 1) and np.all(out2["nev"] == 0)
    st2 = o.state()
    np.testing.assert_array_equal(st2["beta"], st["beta"])
    np.testing.assert_array_equal(st2["xc"], st["xc"])
    np.testing.assert_array_equal(st2["l_last"], st["l_last"])


def test_constant_and_shift():
    """Constant y gives alpha = const, beta = 0 for any ridge; adding k to y
    shifts alpha by k and leaves beta (ridge acts on beta only)."""
    rng = np.random.default_rng(2)
    r, T, H, W = 3, 2, 10, 10
    frames = [(_random_features(rng, H, W), rng.normal(size=(H, W))) for _ in range(T)]
    for ridge in (1e-4, 1e-1):
        o = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=0, mode=EXHAUSTIVE, ridge=ridge))
        o2 = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=0, mode=EXHAUSTIVE, ridge=ridge))
        o3 = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=0, mode=EXHAUSTIVE, ridge=ridge))
        for (n, a, d), y in frames:
            o.push(frame(np.full((H, W), -1.25), n, a, d))
            o2.push(frame(y, n, a, d))
            o3.push(frame(y + 0.75, n, a, d))
        for c in [(5, 5), (0, 9), (9, 0)]:
            th, _, _ = o.wlr_at(*c)
            assert th[0] == pytest.approx(-1.25, abs=1e-12)
            np.testing.assert_allclose(th[1:], 0, atol=1e-12)
            t2, _, _ = o2.wlr_at(*c)
            t3, _, _ = o3.wlr_at(*c)
            assert t3[0] - t2[0] == pytest.approx(0.75, abs=1e-6)  # float32 input rounding
            np.testing.assert_allclose(t3[1:], t2[1:], atol=1e-6)


def _design(frames, cx, cy, r, T, t, h=1.0, bw=(1.0,) * 7):
    """Weighted ridge least squares in matrix form (independent of the oracle)."""
    H, W = frames[0][0].shape
    rows, ys, ws = [], [], []
    fc = frames[t][1][:, cy, cx]
    hb = np.array([h, h] + [h * b for b in bw])
    for tau in range(max(0, t - T + 1), t + 1):
        y, f = frames[tau]
        for qy in range(max(0, cy - r), min(H, cy + r + 1)):
            for qx in range(max(0, cx - r), min(W, cx + r + 1)):
                d = np.concatenate([[(qx - cx) / r, (qy - cy) / r], f[:, qy, qx] - fc])
                ws.append(np.exp(-0.5 * np.sum((d / hb) ** 2)))
                rows.append(np.concatenate([[1.0], d]))
                ys.append(y[qy, qx])
    return np.array(rows), np.array(ys), np.array(ws)


@pytest.mark.parametrize("r,T", [(1, 1), (1, 2), (3, 3)])
def test_matches_numpy_lstsq(r, T):
    """The regression equals numpy's least-squares solve of the sqrt(w)-weighted
    system stacked on sqrt(lambda W) [0 | I] (a library routine, not the
    oracle's QR)."""
    rng = np.random.default_rng(3 + r + T)
    H, W = 2 * r + 4, 2 * r + 5
    lam = 1e-3
    o = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=0, mode=EXHAUSTIVE, ridge=lam))
    frames = []
    for _ in range(T + 1):
        n, a, d = _random_features(rng, H, W)
        y = rng.normal(size=(H, W)).astype(np.float32)
        o.push(frame(y, n, a, d))
        frames.append((y.astype(np.float64), _feat_stack(n, a, d)))
    t = len(frames) - 1
    for cx, cy in [(W // 2, H // 2), (0, 0), (W - 1, 1)]:
        Z, yv, wv = _design(frames, cx, cy, r, T, t)
        Wsum = wv.sum()
        A = np.vstack([np.sqrt(wv)[:, None] * Z, np.sqrt(lam * Wsum) * np.eye(10)[1:]])
        b = np.concatenate([np.sqrt(wv) * yv, np.zeros(9)])
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        theta, R, Wo = o.wlr_at(cx, cy)
        np.testing.assert_allclose(theta, ref, rtol=1e-9, atol=1e-10)
        assert Wo == pytest.approx(Wsum, rel=1e-12)
        assert R == pytest.approx(np.sum(wv * (yv - Z @ ref) ** 2) / Wsum, rel=1e-9)


# ---------------------------------------------------------------- log brightness

def test_log_luminance():
    """y = ln(Y + eps) with Rec.709 luminance for RGB (Section 1.1: L = log E)."""
    H = W = 7
    n, a, d = uniform_features(H, W)
    o = Oracle(OracleConfig(W, H, radius=1, frames=1, channels=1, mode=EXHAUSTIVE, log_eps=1e-3))
    o.push(frame(np.full((H, W), 0.5), n, a, d))
    assert o.wlr_at(3, 3)[0][0] == pytest.approx(math.log(0.5 + 1e-3), abs=1e-12)
    o3 = Oracle(OracleConfig(W, H, radius=1, frames=1, channels=3, mode=EXHAUSTIVE, log_eps=1e-3))
    rgb = np.stack([np.full((H, W), v) for v in (0.25, 0.5, 2.0)])
    o3.push(frame(rgb, n, a, d))
    Y = 0.2126 * 0.25 + 0.7152 * 0.5 + 0.0722 * 2.0
    assert o3.wlr_at(3, 3)[0][0] == pytest.approx(math.log(Y + 1e-3), abs=1e-7)


# ---------------------------------------------------------------- Proposition 1 (Eqs. 6-9)

def test_prop1_identity_literal_residual():
    """With the model kept from the last event, the literal shifted residual of
    Eq. 7 over that event's window minus R equals (beta^T (x^c - xhat^c))^2
    exactly (reading A), because the alpha normal equation makes the weighted
    residuals sum to zero.  The oracle's test statistic is that quantity."""
    rng = np.random.default_rng(4)
    r, T, H, W = 2, 1, 9, 9
    lam = 1e-4
    o = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=0, mode=ADAPTIVE, ridge=lam, contrast=0.2))
    n, a, d = _random_features(rng, H, W)
    y = rng.normal(size=(H, W)).astype(np.float32)
    o.push(frame(y, n, a, d))
    f0 = [(y.astype(np.float64), _feat_stack(n, a, d))]
    cx, cy = 4, 4
    theta, R, _ = o.wlr_at(cx, cy)
    # next frame: only the centre pixel's features move
    n2, a2, d2 = n.copy(), a.copy(), d.copy()
    n2[:, cy, cx] += [0.05, -0.1, 0.02]
    d2[cy, cx] += 0.3
    a2[:, cy, cx] -= [0.1, 0.0, 0.05]
    o.push(frame(y, n2, a2, d2))
    stat = o.outputs()["stat"][cy, cx]
    Z, yv, wv = _design(f0, cx, cy, r, T, 0)
    xc = f0[0][1][:, cy, cx]
    xhat = _feat_stack(n2, a2, d2)[:, cy, cx]
    beta_f = theta[3:]
    # literal Eq. 7: residual of the translated hyperplane over the old window
    shift = beta_f @ (xc - xhat)
    resid_hat = yv - theta[0] - Z[:, 1:] @ theta[1:] - shift
    R_hat = np.sum(wv * resid_hat ** 2) / wv.sum()
    assert R_hat - R == pytest.approx(stat ** 2, rel=1e-10)
    assert stat == pytest.approx(shift, rel=1e-12)


@pytest.mark.parametrize("delta,flag", [(0.25, 1), (0.15, 0), (-0.3, 1)])
def test_flag_threshold_closed_form(delta, flag):
    """Frame 0 fits y = a + g*depth (beta_depth = g).  Moving only the centre's
    depth by delta gives stat = beta^T(x^c - xhat^c) = -g*delta; the pixel is
    flagged iff stat^2 >= C^2, and the new fit moves alpha by g*delta."""
    rng = np.random.default_rng(5)
    r, H, W, g, C = 2, 9, 9, 1.0, 0.2
    o = Oracle(OracleConfig(W, H, radius=r, frames=1, channels=0, mode=ADAPTIVE, ridge=1e-12, contrast=C))
    n, a, _ = uniform_features(H, W)
    d = rng.uniform(2.0, 3.0, (H, W)).astype(np.float32).astype(np.float64)
    o.push(frame(0.1 + g * d, n, a, d))
    d2 = d.copy()
    d2[4, 4] += delta
    o.push(frame(0.1 + g * d2, n, a, d2))
    out = o.outputs()
    assert out["stat"][4, 4] == pytest.approx(-g * delta, abs=1e-5)
    assert out["flag"][4, 4] == flag
    assert out["flag"].sum() == flag          # nothing else moved
    ev = o.take_events()
    if flag:
        assert out["dl"][4, 4] == pytest.approx(g * delta, abs=1e-5)
        k = int(math.floor(abs(g * delta) / C + 1e-9))
        assert len(ev) == k and all(e[3] == np.sign(delta) for e in ev)
    else:
        assert len(ev) == 0


# ---------------------------------------------------------------- events (Eq. 1)

def test_static_noise_free_scene_no_events():
    """A static, noise-free scene never changes brightness: no events in either mode."""
    from scenes import Scene, preset
    s = Scene(preset("disc64", disc_velocity=(0.0, 0.0)))
    c = s.clean(0)
    fr = {"radiance": c["radiance"].float().numpy(), "normal": c["normal"].float().numpy(),
          "albedo": c["albedo"].float().numpy(), "depth": c["depth"].float().numpy()}
    for mode in (ADAPTIVE, EXHAUSTIVE):
        o = Oracle(OracleConfig(64, 64, radius=3, frames=3, channels=1, mode=mode, contrast=0.2))
        for _ in range(6):
            o.push(fr)
        assert len(o.take_events()) == 0


def _load_step_golden():
    import json
    import os
    p = os.path.join(os.path.dirname(__file__), "golden", "global_step_T3_C0.2.json")
    with open(p) as f:
        return json.load(f)


def test_global_step_closed_form_events():
    """Static scene, radiance multiplied by e^s from frame k on (exhaustive):
    design rows repeat across frames, so alpha_{k+m} = alpha + s*min(m+1,T)/T;
    with T=3, C=0.2, s=ln 2 every pixel fires once at k, k+1, k+2 (Eq. 1)."""
    gold = _load_step_golden()
    T, C, k = gold["T"], gold["C"], gold["k"]
    s_log = math.log(gold["gain"])
    from scenes import Scene, preset
    sc = Scene(preset("disc64", disc_velocity=(0.0, 0.0)))
    c = sc.clean(0)
    base = {"normal": c["normal"].float().numpy(), "albedo": c["albedo"].float().numpy(),
            "depth": c["depth"].float().numpy()}
    y0 = np.log(c["radiance"][0].double().numpy() + 1e-3)
    H, W = y0.shape
    for mode, expect in ((EXHAUSTIVE, gold["events_per_pixel_by_frame"]), (ADAPTIVE, None)):
        o = Oracle(OracleConfig(W, H, radius=3, frames=T, channels=0, mode=mode, contrast=C))
        per_frame = []
        for t in range(k + 5):
            y = y0 + (s_log if t >= k else 0.0)
            o.push(dict(base, radiance=y.astype(np.float32)))
            ev = o.take_events()
            per_frame.append(len(ev))
            if mode == EXHAUSTIVE and t >= k and len(ev):
                assert np.all(ev[:, 3] == 1)
                dl = o.outputs()["dl"]
                m = t - k
                assert np.allclose(dl[np.isfinite(dl)], gold["dl_by_frame"][m], atol=1e-5)
        if expect is None:
            assert sum(per_frame) == 0      # features static: Prop. 1 never flags
        else:
            assert per_frame == [H * W * e for e in expect]


def test_global_step_with_variance_guard():
    """The optional guard flags a pixel whose log brightness moved by at least
    C + kappa * sigma_y since its last event.  On the global step the guard
    alone lets the adaptive mode fire, and then every flagged pixel regresses
    exactly the exhaustive window, so the events equal the closed-form
    exhaustive ones; with a noise deviation larger than the step the guard
    stays silent (sigma_y = sqrt(Var[Y]) / (Y + eps), Y + eps = e^y)."""
    gold = _load_step_golden()
    T, C, k = gold["T"], gold["C"], gold["k"]
    s_log = math.log(gold["gain"])
    from scenes import Scene, preset
    sc = Scene(preset("disc64", disc_velocity=(0.0, 0.0)))
    c = sc.clean(0)
    base = {"normal": c["normal"].float().numpy(), "albedo": c["albedo"].float().numpy(),
            "depth": c["depth"].float().numpy()}
    y0 = np.log(c["radiance"][0].double().numpy() + 1e-3)
    H, W = y0.shape
    for var_scale, expect in ((0.0, gold["events_per_pixel_by_frame"]), (4.0, [0] * (k + 5))):
        o = Oracle(OracleConfig(W, H, radius=3, frames=T, channels=0, mode=ADAPTIVE, contrast=C, guard_kappa=3.0))
        per_frame = []
        for t in range(k + 5):
            y = y0 + (s_log if t >= k else 0.0)
            # Var[Y] = (var_scale (Y + eps))^2: sigma_y = var_scale, kappa sigma_y = 12 > s
            var = (var_scale * np.exp(y)) ** 2
            o.push(dict(base, radiance=y.astype(np.float32), variance=var.astype(np.float32)))
            per_frame.append(len(o.take_events()))
        assert per_frame == [H * W * e for e in expect]


@pytest.mark.parametrize("jump,C,n_exp", [(1.1, 0.2, 5), (-0.5, 0.2, -2), (0.19, 0.2, 0), (0.2, 0.1, 2)])
def test_multiple_crossings_and_reference_update(jump, C, n_exp):
    """n = floor(|dL|/C) events of polarity sign(dL); L_last moves by p*n*C, so
    the remainder carries over to the next frame."""
    H = W = 5
    n, a, d = uniform_features(H, W)
    o = Oracle(OracleConfig(W, H, radius=1, frames=1, channels=0, mode=EXHAUSTIVE, contrast=C))
    o.push(frame(np.zeros((H, W)), n, a, d))
    o.push(frame(np.full((H, W), jump, np.float32), n, a, d))
    out = o.outputs()
    assert np.all(out["nev"] == n_exp)
    ev = o.take_events()
    assert len(ev) == H * W * abs(n_exp)
    # canonical order: row-major pixels, repeats adjacent
    if len(ev):
        assert np.all(np.diff(ev[:, 2] * W + ev[:, 1]) >= 0)
    l_last = o.state()["l_last"]
    assert np.allclose(l_last, n_exp * C, atol=1e-12)
    y1 = float(np.float32(jump))
    remainder = y1 - n_exp * C
    o.push(frame(np.full((H, W), jump, np.float32), n, a, d))
    assert np.all(o.outputs()["dl"] == pytest.approx(remainder, abs=1e-12))
