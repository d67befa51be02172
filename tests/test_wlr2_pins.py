"""Pins of the second-order regression oracle (oracle/wlr2.py) against facts
that the definitions fix: the closed-form centre weights of a weighted
quadratic fit on a symmetric grid (Savitzky-Golay with Gaussian weights),
exact reproduction of a quadratic field, the weighted mean as the ridge grows
without bound, shift and constant invariants, and an independent solve of the
normal equations on tiny inputs with clipped windows."""
import itertools

import numpy as np
import pytest

from oracle import wlr2 as O


def _flat_features(F, H, W):
    f = np.zeros((F, 7, H, W))
    f[:, 2] = 1.0     # normal (0, 0, 1)
    f[:, 3] = 2.0     # depth
    f[:, 4:] = 0.5    # albedo
    return f


def _centre_weights_1d(r, h):
    """Weight of sample i in the value at 0 of a Gaussian-weighted fit of
    {1, x^2} (the odd terms drop out on a symmetric grid), x = i / r."""
    x = np.arange(-r, r + 1) / r
    g = np.exp(-0.5 * (x / h) ** 2)
    G0, G2, G4 = g.sum(), (g * x ** 2).sum(), (g * x ** 4).sum()
    return g, g * (G4 - G2 * x ** 2) / (G0 * G4 - G2 ** 2)


@pytest.mark.parametrize("T,h", [(1, 1.0), (2, 1.0), (1, 0.7)])
def test_weighted_savitzky_golay_centre(T, h):
    """Constant features: only the coordinate terms (1, x, y, x^2, xy, y^2)
    remain, with separable weights g_i g_j.  On the tensor grid the projection
    onto {1, x^2, y^2} is P_U x P_1 + P_1 x P_U - P_1 x P_1 (U = span{1, x^2}),
    so the centre value is sum_ij c_ij ybar_ij with
    c_ij = a_i g_j / G0 + g_i a_j / G0 - g_i g_j / G0^2; ybar averages the T
    frames, whose design rows coincide."""
    r, F, H, W = 3, 3, 12, 14
    rng = np.random.default_rng(5)
    rad = rng.uniform(0.1, 3.0, size=(F, 1, H, W))
    alpha = O.wlr2(rad, _flat_features(F, H, W), radius=r, frames=T, h=h, ridge=1e-12)
    y = O.log_brightness(rad, 1e-3)
    g, a = _centre_weights_1d(r, h)
    G0 = g.sum()
    c = np.outer(g / G0, a) + np.outer(a, g / G0) - np.outer(g / G0, g / G0)
    t = F - 1
    ybar = y[t - T + 1:t + 1].mean(axis=0)
    for cy in range(r, H - r):
        for cx in range(r, W - r):
            ref = float((c * ybar[cy - r:cy + r + 1, cx - r:cx + r + 1]).sum())
            assert alpha[t, cy, cx] == pytest.approx(ref, abs=1e-9)


def test_one_row_image_is_the_1d_fit():
    r, W = 4, 17
    rng = np.random.default_rng(2)
    rad = rng.uniform(0.1, 3.0, size=(1, 1, 1, W))
    alpha = O.wlr2(rad, _flat_features(1, 1, W), radius=r, frames=1, ridge=1e-12)
    y = O.log_brightness(rad, 1e-3)[0, 0]
    _, a = _centre_weights_1d(r, 1.0)
    for cx in range(r, W - r):
        assert alpha[0, 0, cx] == pytest.approx(float(a @ y[cx - r:cx + r + 1]), abs=1e-10)


def test_quadratic_field_is_reproduced():
    """y = c0 + g^T x + x^T Q x in the absolute 9-D feature is quadratic in
    d = x - x^c, so the fit has zero residual and alpha is y at the centre.
    Random features keep the 55 columns independent; only centres whose window
    holds well over 55 samples are checked (a smaller window fits any y), so a
    dropped or wrong cross term breaks this."""
    rng = np.random.default_rng(11)
    F, H, W, r, T = 3, 10, 11, 3, 2
    feat = rng.uniform(-1.0, 1.0, size=(F, 7, H, W))
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    X = np.concatenate([np.broadcast_to((xx / r)[None, None], (F, 1, H, W)),
                        np.broadcast_to((yy / r)[None, None], (F, 1, H, W)), feat], axis=1)   # [F][9][H][W]
    g = rng.normal(size=9)
    Q = rng.normal(size=(9, 9)) * 0.3
    y = 0.4 + np.einsum("j,fjhw->fhw", g, X) + np.einsum("jk,fjhw,fkhw->fhw", Q, X, X)
    eps = 1e-3
    rad = (np.exp(y) - eps)[:, None]
    alpha = O.wlr2(rad, feat, radius=r, frames=T, ridge=1e-13, log_eps=eps)
    n_side = lambda c, n: min(n, c + r + 1) - max(0, c - r)
    checked = 0
    cen = []
    for t, cy, cx in itertools.product(range(1, F), range(H), range(W)):
        if n_side(cy, H) * n_side(cx, W) * T >= 80:
            assert alpha[t, cy, cx] == pytest.approx(y[t, cy, cx], abs=1e-7)
            checked += 1
            if cx != cy:
                cen.append((t, cy, cx))
    assert checked > 50
    # the listed-centres path, (t, y, x) per centre, reproduces the field too
    cen = cen[::3]
    a_c = O.wlr2(rad, feat, radius=r, frames=T, ridge=1e-13, log_eps=eps, centres=cen)
    np.testing.assert_allclose(a_c, [y[t, cy, cx] for t, cy, cx in cen], rtol=0, atol=1e-7)


def test_infinite_ridge_gives_the_weighted_mean():
    """As lambda grows every coefficient but the intercept goes to zero and
    alpha becomes sum w y / W with the product-Gaussian weights of Eq. 5; this
    pins the weights, feature bandwidths included."""
    rng = np.random.default_rng(4)
    F, H, W, r, T = 2, 6, 7, 2, 2
    feat = rng.uniform(0.0, 1.0, size=(F, 7, H, W))
    rad = rng.uniform(0.2, 2.0, size=(F, 3, H, W))
    b = (0.5, 1.0, 2.0, 0.8, 1.3, 0.6, 1.1)
    h = 0.9
    alpha = O.wlr2(rad, feat, bandwidth=b, radius=r, frames=T, h=h, ridge=1e14)
    y = O.log_brightness(rad, 1e-3)
    hb = np.array([h, h] + [h * v for v in b])
    t = F - 1
    for cy, cx in itertools.product(range(H), range(W)):
        num = den = 0.0
        for tau in range(max(0, t - T + 1), t + 1):
            for qy in range(max(0, cy - r), min(H, cy + r + 1)):
                for qx in range(max(0, cx - r), min(W, cx + r + 1)):
                    d = np.concatenate([[(qx - cx) / r, (qy - cy) / r], feat[tau, :, qy, qx] - feat[t, :, cy, cx]])
                    w = np.exp(-0.5 * np.sum((d / hb) ** 2))
                    num += w * y[tau, qy, qx]
                    den += w
        assert alpha[t, cy, cx] == pytest.approx(num / den, abs=1e-8)


def test_shift_and_constant_invariants():
    rng = np.random.default_rng(8)
    F, H, W = 2, 7, 8
    feat = rng.uniform(0.0, 1.0, size=(F, 7, H, W))
    rad = rng.uniform(0.2, 2.0, size=(F, 1, H, W))
    eps, k = 1e-3, 0.75
    a0 = O.wlr2(rad, feat, radius=2, frames=2, log_eps=eps)
    a1 = O.wlr2((rad + eps) * np.exp(k) - eps, feat, radius=2, frames=2, log_eps=eps)
    np.testing.assert_allclose(a1, a0 + k, rtol=0, atol=1e-10)
    const = O.wlr2(np.full((F, 1, H, W), 0.37), feat, radius=2, frames=2, log_eps=eps)
    np.testing.assert_allclose(const, np.log(0.37 + eps), rtol=0, atol=1e-12)


def test_normal_equations_on_clipped_windows():
    """An independent solver: the 55 x 55 normal equations (Z^T W Z + lambda W P)
    theta = Z^T W y in plain loops, on an image smaller than the window."""
    rng = np.random.default_rng(21)
    F, H, W, r, T = 3, 4, 5, 3, 2
    feat = rng.uniform(0.0, 1.0, size=(F, 7, H, W))
    rad = rng.uniform(0.2, 2.0, size=(F, 3, H, W))
    lam = 1e-3
    alpha = O.wlr2(rad, feat, radius=r, frames=T, ridge=lam)
    y = O.log_brightness(rad, 1e-3)
    pairs = [(a, b) for a in range(9) for b in range(a, 9)]
    for t, cy, cx in itertools.product(range(F), range(H), range(W)):
        A = np.zeros((55, 55))
        rhs = np.zeros(55)
        Wsum = 0.0
        for tau in range(max(0, t - T + 1), t + 1):
            for qy in range(H):
                for qx in range(W):
                    if abs(qx - cx) > r or abs(qy - cy) > r:
                        continue
                    d = np.concatenate([[(qx - cx) / r, (qy - cy) / r], feat[tau, :, qy, qx] - feat[t, :, cy, cx]])
                    w = np.exp(-0.5 * np.sum(d ** 2))
                    z = np.concatenate([[1.0], d, [d[a] * d[b] for a, b in pairs]])
                    A += w * np.outer(z, z)
                    rhs += w * y[tau, qy, qx] * z
                    Wsum += w
        A[np.arange(1, 55), np.arange(1, 55)] += lam * Wsum
        assert alpha[t, cy, cx] == pytest.approx(np.linalg.solve(A, rhs)[0], abs=1e-9)


def test_agrees_with_the_first_order_oracle_where_both_are_exact():
    """Two independent oracles, one window and weight convention: on a field
    linear in the 9-D feature both fits are exact (same alpha as y at the
    centre), and as the ridge grows both become the same weighted mean.  This
    ties the second-order oracle's windows (clipping, causal frames), coordinate
    units and weights to the first-order C oracle."""
    from oracle import EXHAUSTIVE, Oracle, OracleConfig
    rng = np.random.default_rng(13)
    F, H, W, r, T = 3, 8, 9, 2, 2
    feat = rng.uniform(0.0, 1.0, size=(F, 7, H, W)).astype(np.float32).astype(np.float64)
    rad_w = rng.uniform(0.2, 2.0, size=(F, 1, H, W)).astype(np.float32).astype(np.float64)
    b = [0.7, 1.3, 0.9, 1.6, 0.8, 1.2, 1.0]

    def first_order(rad, ridge):
        o = Oracle(OracleConfig(W, H, radius=r, frames=T, channels=rad.shape[1], mode=EXHAUSTIVE, bandwidth=b,
                                ridge=ridge))
        out = []
        for t in range(F):
            o.push({"radiance": rad[t].astype(np.float32), "normal": feat[t, 0:3].astype(np.float32),
                    "depth": feat[t, 3].astype(np.float32), "albedo": feat[t, 4:7].astype(np.float32)})
            out.append(o.outputs()["alpha"])
        return np.stack(out)

    a1 = first_order(rad_w, 1e14)
    a2 = O.wlr2(rad_w, feat, bandwidth=b, radius=r, frames=T, ridge=1e14)
    np.testing.assert_allclose(a2, a1, rtol=0, atol=1e-9)
    # RGB radiance: each oracle forms its own Rec.709 luminance
    rad_rgb = rng.uniform(0.2, 2.0, size=(F, 3, H, W)).astype(np.float32).astype(np.float64)
    a1 = first_order(rad_rgb, 1e14)
    a2 = O.wlr2(rad_rgb, feat, bandwidth=b, radius=r, frames=T, ridge=1e14)
    np.testing.assert_allclose(a2, a1, rtol=0, atol=1e-9)
    # a field linear in the feature: both reproduce it (to the float32 rounding of the radiance)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    g = rng.normal(size=9)
    lin = (0.3 + g[0] * xx / r + g[1] * yy / r)[None] + np.einsum("j,fjhw->fhw", g[2:], feat)
    rad_l = (np.exp(lin) - 1e-3)[:, None].astype(np.float32).astype(np.float64)
    y_l = O.log_brightness(rad_l, 1e-3)
    a1 = first_order(rad_l, 1e-12)
    a2 = O.wlr2(rad_l, feat, bandwidth=b, radius=r, frames=T, ridge=1e-12)
    np.testing.assert_allclose(a1, y_l, rtol=0, atol=2e-6)
    np.testing.assert_allclose(a2, y_l, rtol=0, atol=2e-6)
