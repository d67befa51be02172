"""FP64 reference of the differentiable dense regression, for the tests.

A plain torch restatement of Eqs. 3-5 (with the ridge lambda W |beta|^2 on the
slopes), vectorised over the centres of a small crop, solved either by
torch.linalg.solve on the weighted normal equations or by torch.linalg.lstsq
on the sqrt(w)-weighted design stacked on the ridge rows sqrt(lambda W) [0 | I]
(the dense least-squares form), so that torch autograd gives the reference
gradients in double precision.  It shares no code with the CUDA library; its
gradients are pinned against central finite differences of the FP64 oracle
in test_adjoint_pins.py.
"""
from __future__ import annotations

import torch

REC709 = (0.2126, 0.7152, 0.0722)


def log_luminance(rad: torch.Tensor, eps: float) -> torch.Tensor:
    """rad [F][C][H][W] -> y [F][H][W] = ln(Y + eps)."""
    Y = rad[:, 0] if rad.shape[1] == 1 else sum(w * rad[:, i] for i, w in enumerate(REC709))
    return torch.log(Y + eps)


def wlr_alpha(rad, feat, b, r: int, T: int, h: float = 1.0, eps: float = 1e-3, ridge: float = 1e-4,
              solver: str = "solve"):
    """alpha [F][H][W] of every pixel and frame (window frames t-T+1..t, clipped);
    solver "solve" (normal equations) or "lstsq" (augmented least squares)."""
    F, _, H, W = rad.shape
    y = log_luminance(rad, eps)                                     # [F][H][W]
    dt = rad.dtype
    side = 2 * r + 1
    yp = torch.nn.functional.pad(y, (r, r, r, r))
    fp = torch.nn.functional.pad(feat, (r, r, r, r))
    valid = torch.nn.functional.pad(torch.ones(H, W, dtype=dt), (r, r, r, r))
    hb = torch.cat([torch.full((2,), h, dtype=dt), h * b])          # bandwidths of the 9 regressors
    P = torch.diag(torch.tensor([0.0] + [1.0] * 9, dtype=dt))
    out = []
    for t in range(F):
        Zs, ys, ws = [], [], []
        xc = feat[t]                                                 # [7][H][W]
        for tau in range(max(0, t - T + 1), t + 1):
            for oy in range(-r, r + 1):
                for ox in range(-r, r + 1):
                    sl = (slice(r + oy, r + oy + H), slice(r + ox, r + ox + W))
                    d = torch.cat([torch.full((2, H, W), 0.0, dtype=dt), fp[tau][(slice(None),) + sl] - xc], 0)
                    d[0] = ox / r
                    d[1] = oy / r
                    # sqrt(w) directly (no sqrt of w = 0 at clipped offsets)
                    sw = torch.exp(-0.25 * (((d / hb.view(9, 1, 1)) ** 2).sum(0))) * valid[sl]
                    Zs.append(torch.cat([torch.ones(1, H, W, dtype=dt), d], 0))
                    ys.append(yp[tau][sl])
                    ws.append(sw)
        Z = torch.stack(Zs, -1).permute(1, 2, 3, 0)                  # [H][W][K][10]
        yv = torch.stack(ys, -1)                                     # [H][W][K]
        sw = torch.stack(ws, -1)                                     # [H][W][K] sqrt(w)
        wv = sw * sw
        if solver == "lstsq":
            Wsum = wv.sum(-1)
            ridge_rows = torch.sqrt(ridge * Wsum)[..., None, None] * P[1:].expand(H, W, 9, 10)
            M = torch.cat([sw[..., None] * Z, ridge_rows], -2)       # [H][W][K+9][10]
            rhs = torch.cat([sw * yv, torch.zeros(H, W, 9, dtype=dt)], -1)
            theta = torch.linalg.lstsq(M, rhs.unsqueeze(-1)).solution.squeeze(-1)
        else:
            A = torch.einsum("hwk,hwki,hwkj->hwij", wv, Z, Z) + ridge * wv.sum(-1)[..., None, None] * P
            g = torch.einsum("hwk,hwk,hwki->hwi", wv, yv, Z)
            theta = torch.linalg.solve(A, g.unsqueeze(-1)).squeeze(-1)
        out.append(theta[..., 0])
    return torch.stack(out, 0)


def mse_loss(alpha, clean, eps: float = 1e-3):
    """Mean over pixels and frames of (alpha - ln(Y_clean + eps))^2."""
    return ((alpha - log_luminance(clean, eps)) ** 2).mean()
