"""FP64 oracle of the second-order weighted local regression.

TEST INFRASTRUCTURE ONLY: the independent reference that the library's
second-order kernel is checked against.  Only the tests and the benchmark's
CPU-baseline leg use it; the library never does.  Plain numpy in float64.

What it computes.  Eq. 3 approximates the unknown log brightness f around the
centre feature x^c by its first-order Taylor expansion, and Eqs. 4-5 fit that
expansion by Gaussian-weighted least squares over the window Omega_c.  The
paper's conclusion (Section 4) names a non-linear regression as the natural
extension.  Here the expansion is carried one order further:

    f(x) ~ alpha + beta^T d + sum_{a <= b} gamma_ab d_a d_b,   d = x - x^c,

so the design row of neighbour i is z^i = (1, d^i, [d^i_a d^i_b]_{a<=b}) with
1 + 9 + 45 = 55 entries over the 9-D feature (coordinate offset (q - c)/r,
normal, depth, albedo).  The weights are those of Eq. 5 (product Gaussian,
coordinate bandwidths h, feature bandwidths h b_j); the window is the spatial
square |q - c|_inf <= r clipped to the image over the causal frames
max(0, t - T + 1) .. t.  Minimise

    sum_i w^i (y^i - theta^T z^i)^2 + lambda W sum_{k >= 1} theta_k^2

(the ridge covers every coefficient but the intercept, in the natural units of
z, as the first-order simulator does for beta) and output alpha = theta_0, the
denoised log brightness at the centre.  The solve is a Householder QR of the
sqrt(w)-weighted design stacked on sqrt(lambda W) [0 | I_54].
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

LUMA = np.array([0.2126, 0.7152, 0.0722])
ND = 9                                     # dx, dy, normal xyz, depth, albedo rgb
PAIRS = [(a, b) for a in range(ND) for b in range(a, ND)]
NZ = 1 + ND + len(PAIRS)                   # 55 unknowns


def log_brightness(radiance: np.ndarray, log_eps: float) -> np.ndarray:
    """y = ln(Y + eps) per frame, Y the Rec.709 luminance of RGB input (or the
    single channel itself).  radiance [F][C][H][W] -> [F][H][W] float64."""
    r = np.asarray(radiance, dtype=np.float64)
    Y = r[:, 0] if r.shape[1] == 1 else np.tensordot(LUMA, r, axes=([0], [1]))
    return np.log(Y + log_eps)


def design_row(d: np.ndarray) -> np.ndarray:
    """z = (1, d, d_a d_b for a <= b) for offsets d [..., 9] -> [..., 55]."""
    quad = np.stack([d[..., a] * d[..., b] for a, b in PAIRS], axis=-1)
    return np.concatenate([np.ones(d.shape[:-1] + (1,)), d, quad], axis=-1)


def _window(y, feat, t, cx, cy, radius, frames):
    """Offsets d [P][M][9], log brightness [P][M] and a validity mask [P][M] of
    the windows of centres (cx, cy) in frame t; M = (2r+1)^2 * frames."""
    F, _, H, W = feat.shape
    offs = np.arange(-radius, radius + 1)
    taus = np.arange(t - frames + 1, t + 1)
    tt, oy, ox = np.meshgrid(taus, offs, offs, indexing="ij")
    tt, oy, ox = tt.ravel(), oy.ravel(), ox.ravel()
    qx = cx[:, None] + ox[None, :]
    qy = cy[:, None] + oy[None, :]
    tq = np.broadcast_to(tt[None, :], qx.shape)
    valid = (qx >= 0) & (qx < W) & (qy >= 0) & (qy < H) & (tq >= 0)
    qxc, qyc, tqc = np.clip(qx, 0, W - 1), np.clip(qy, 0, H - 1), np.clip(tq, 0, F - 1)
    xq = feat[tqc, :, qyc, qxc]                       # [P][M][7]
    xc = feat[t, :, cy, cx]                           # [P][7]
    d = np.empty(qx.shape + (ND,))
    d[..., 0] = (qx - cx[:, None]) / radius
    d[..., 1] = (qy - cy[:, None]) / radius
    d[..., 2:] = xq - xc[:, None, :]
    return d, y[tqc, qyc, qxc], valid


def _solve(d, yv, valid, hb, ridge):
    """alpha = theta_0 of the ridged weighted least squares, one per centre.
    The right-hand side rides along as a 56th column, so the Householder
    triangularisation of [A | b] leaves R and Q^T b side by side."""
    w = np.exp(-0.5 * np.sum((d / hb) ** 2, axis=-1)) * valid          # Eq. 5
    W = w.sum(axis=1)
    sw = np.sqrt(w)
    data = np.concatenate([sw[..., None] * design_row(d), (sw * yv)[..., None]], axis=-1)   # [P][M][56]
    ridge_rows = np.zeros((d.shape[0], NZ - 1, NZ + 1))
    ridge_rows[:, np.arange(NZ - 1), np.arange(1, NZ)] = np.sqrt(ridge * W)[:, None]
    aug = np.concatenate([data, ridge_rows], axis=1)
    alpha = np.empty(d.shape[0])
    for p in range(d.shape[0]):
        R = scipy.linalg.qr(aug[p], mode="r", check_finite=False)[0]       # LAPACK dgeqrf
        theta = scipy.linalg.solve_triangular(R[:NZ, :NZ], R[:NZ, NZ])
        alpha[p] = theta[0]
    return alpha


def wlr2(radiance, features, bandwidth=(1.0,) * 7, radius: int = 3, frames: int = 3, h: float = 1.0,
         log_eps: float = 1e-3, ridge: float = 1e-4, centres=None, chunk_bytes: int = 64 << 20):
    """Second-order regression of every pixel of every frame (or of the listed
    centres (t, y, x)).  radiance [F][C][H][W], features [F][7][H][W] (normal
    xyz, depth, albedo rgb).  Returns alpha [F][H][W] (or [len(centres)]) in
    float64."""
    feat = np.asarray(features, dtype=np.float64)
    y = log_brightness(radiance, log_eps)
    F, _, H, W = feat.shape
    hb = np.array([h, h] + [h * float(b) for b in bandwidth])
    M = (2 * radius + 1) ** 2 * frames
    per = max(1, chunk_bytes // ((M + NZ) * (NZ + 1) * 8 * 3))
    if centres is None:
        out = np.empty((F, H, W))
        for t in range(F):
            cy, cx = np.divmod(np.arange(H * W), W)
            flat = out[t].reshape(-1)
            for s in range(0, H * W, per):
                d, yv, valid = _window(y, feat, t, cx[s:s + per], cy[s:s + per], radius, frames)
                flat[s:s + per] = _solve(d, yv, valid, hb, ridge)
        return out
    cen = np.asarray(centres, dtype=np.int64).reshape(-1, 3)
    out = np.empty(len(cen))
    for t in np.unique(cen[:, 0]):
        idx = np.nonzero(cen[:, 0] == t)[0]
        for s in range(0, len(idx), per):
            k = idx[s:s + per]
            d, yv, valid = _window(y, feat, int(t), cen[k, 2], cen[k, 1], radius, frames)
            out[k] = _solve(d, yv, valid, hb, ridge)
    return out
