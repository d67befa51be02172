"""FP64 CPU oracle of the event-quality evaluation (Section 3, quantitative
comparison).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the CUDA evaluation
kernels are checked against it; the library never uses it.

- ``esim_counts``: the plain ESIM simulator the paper compares with (and whose
  run on noise-free frames stands in for the paper's 4096-spp reference):
  Eq. 1 applied to the log brightness of each frame itself, with the same
  multiple-crossing rule as the simulator (n = floor(|dL| / C) events of
  polarity sign(dL), L_last += p n C; frame 0 only initialises L_last).
- ``quality``: events as signed points (x, y, t); precision P(tau) counts the
  generated events whose nearest reference event of the same polarity is
  closer than tau, recall R(tau) the reference events whose nearest generated
  event of the same polarity is closer than tau (Eqs. 10a-b), F(tau) their
  harmonic mean, and the polarity-aware chamfer distance the mean squared
  nearest-neighbour distance in both directions.  Coordinates are
  (x / W, y / H, t / F).  Nearest neighbours come from a k-d tree (scipy).
"""
from __future__ import annotations

import numpy as np

REC709 = (0.2126, 0.7152, 0.0722)


def log_brightness(radiance: np.ndarray, eps: float = 1e-3) -> np.ndarray:
    """ln(Y + eps) in FP64; radiance [C][H][W] with C = 1 (luminance) or 3 (RGB)."""
    r = np.asarray(radiance, np.float64)
    Y = r[0] if r.shape[0] == 1 else REC709[0] * r[0] + REC709[1] * r[1] + REC709[2] * r[2]
    return np.log(Y + eps)


def esim_step(y: np.ndarray, l_last: np.ndarray | None, C: float):
    """One frame of plain ESIM: returns (signed counts, new L_last).  With
    l_last None the frame initialises the reference level and emits nothing."""
    y = np.asarray(y, np.float64)
    if l_last is None:
        return np.zeros(y.shape, np.int64), y.copy()
    dl = y - l_last
    n = np.floor(np.abs(dl) / C).astype(np.int64)
    p = np.where(dl >= 0, 1, -1)
    counts = p * n
    return counts, l_last + counts * C


def esim_counts(y_frames, C: float) -> np.ndarray:
    """Signed event counts [F][H][W] of a log-brightness sequence [F][H][W]."""
    out, level = [], None
    for y in y_frames:
        c, level = esim_step(y, level, C)
        out.append(c)
    return np.stack(out)


def event_points(counts: np.ndarray, polarity: int):
    """Points (x/W, y/H, t/F) of the events of one polarity in a signed count
    map [F][H][W], with their multiplicities."""
    F, H, W = counts.shape
    sel = counts * polarity > 0
    t, y, x = np.nonzero(sel)
    pts = np.stack([x / W, y / H, t / F], axis=1).astype(np.float64)
    return pts, np.abs(counts[sel]).astype(np.int64)


def nearest_distances(query: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Euclidean distance from each query point to its nearest reference
    point (inf when there are no reference points)."""
    if len(query) == 0:
        return np.zeros(0)
    if len(ref) == 0:
        return np.full(len(query), np.inf)
    from scipy.spatial import cKDTree
    d, _ = cKDTree(ref).query(query, k=1)
    return np.asarray(d, np.float64)


def directed(query_counts: np.ndarray, ref_counts: np.ndarray):
    """Per-event nearest same-polarity distances from one set to the other:
    (distances, multiplicities) over both polarities."""
    ds, ws = [], []
    for p in (1, -1):
        q, w = event_points(query_counts, p)
        r, _ = event_points(ref_counts, p)
        ds.append(nearest_distances(q, r))
        ws.append(w)
    return np.concatenate(ds), np.concatenate(ws)


def quality(gen: np.ndarray, ref: np.ndarray, taus) -> dict:
    """P(tau), R(tau), F(tau) and the chamfer distance of generated events
    `gen` against reference events `ref` (signed count maps [F][H][W])."""
    dg, wg = directed(gen, ref)
    dr, wr = directed(ref, gen)
    ng, nr = int(wg.sum()), int(wr.sum())
    P, R, Fs = [], [], []
    for tau in taus:
        p = float(wg[dg < tau].sum()) / ng if ng else 0.0
        r = float(wr[dr < tau].sum()) / nr if nr else 0.0
        P.append(p)
        R.append(r)
        Fs.append(2 * p * r / (p + r) if p + r > 0 else 0.0)
    cd = (float((wg * dg ** 2).sum()) / ng if ng else 0.0) + (float((wr * dr ** 2).sum()) / nr if nr else 0.0)
    return {"precision": P, "recall": R, "fscore": Fs, "chamfer": cd, "n_gen": ng, "n_ref": nr,
            "d_gen": dg, "w_gen": wg, "d_ref": dr, "w_ref": wr}
