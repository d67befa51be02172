"""Bandwidth selection: the seven feature bandwidths b_j of the product
Gaussian (Eq. 5) fitted by gradient descent on the differentiation form's loss,
mean over pixels and frames of (alpha - ln(Y_clean + eps))^2, so that the
fitted b can be fed back into the adaptive simulator.  The paper keeps
h = 1, b_j = 1 and reports that per-pixel bandwidth optimisation (after
Moon et al.) costs about 8x the time for little gain (Section 3); this is the
global, learned alternative.

Every forward and backward pass runs the library's dense regression and its
hand-written adjoint (``wlr``); the loop here only updates seven numbers.
"""
from __future__ import annotations

REC709 = (0.2126, 0.7152, 0.0722)


def log_luminance(radiance, eps: float = 1e-3):
    """ln(Y + eps) of radiance [F][C][H][W] (C = 1 or 3)."""
    import torch
    if radiance.shape[1] == 3:
        Y = REC709[0] * radiance[:, 0] + REC709[1] * radiance[:, 1] + REC709[2] * radiance[:, 2]
    else:
        Y = radiance[:, 0]
    return torch.log(Y + eps)


def fit_bandwidths(radiance, features, clean, radius: int = 3, frames: int = 3, steps: int = 60,
                   lr: float = 0.1, b0=None, log_eps: float = 1e-3, ridge: float = 1e-4):
    """Fit b on one training sequence (device tensors: radiance and clean
    [F][C][H][W], features [F][7][H][W]).  b = exp(theta) keeps the
    bandwidths positive; Adam on theta.  Returns (b as a list of floats, loss
    per step)."""
    import torch
    from . import wlr
    dev = radiance.device
    target = log_luminance(clean.float(), log_eps)
    start = torch.ones(7, device=dev) if b0 is None else torch.as_tensor(b0, dtype=torch.float32, device=dev)
    theta = torch.log(start).clone().requires_grad_(True)
    opt = torch.optim.Adam([theta], lr=lr)
    history = []
    for _ in range(steps):
        opt.zero_grad()
        alpha = wlr(radiance, features, torch.exp(theta), radius=radius, frames=frames, log_eps=log_eps,
                    ridge=ridge)
        loss = ((alpha - target) ** 2).mean()
        loss.backward()
        opt.step()
        history.append(float(loss.detach()))
    return [float(v) for v in torch.exp(theta.detach()).cpu()], history
