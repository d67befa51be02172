"""Host-side logic of the strip split of one large sequence over several GPUs.

One process per GPU simulates a horizontal strip of the image: rank k owns
rows [lo_k, hi_k) (the rows split as evenly as possible) and keeps, in its own
ring, r extra rows above and below (the halo) so that every window of an owned
pixel is local.  Per frame the only exchange is the halo of the new frame:
rank k sends its first r owned rows up to rank k-1 and its last r owned rows
down to rank k+1, and receives the neighbours' rows into its halo; the older
frames' halo rows are already in every ring from their own frames.  That is
2 r W pixels of the new frame per internal boundary, as input planes (16 bytes
per pixel in the precision form's FP16/BF16 storage formats, 40 in FP32) or
as ring records (16 or 32 bytes).  The
test, the regression and the emission are pixel-local, so an owned pixel's
results depend on the held rows only; the owned rows' event lists, each in
(row, column, repeat) order, concatenate in rank order into the whole image's
canonical order.

The exchange is written against torch.distributed point-to-point calls (NCCL
between GPUs; gloo on CPU for the tests), on records laid out
[planes][rows][width] with the halo rows first and last.

StripSimulator is one rank's simulator: a context over its held rows, fed
the held rows of each frame (its own rows plus the halo rows that the
exchange delivers), whose results are kept for the owned rows only.  The
halo rows are converted, tested and regressed like the others (their windows
are clipped at the strip's edge, so their results are discarded); that costs
2 r rows of extra work per internal boundary.
"""
from __future__ import annotations


def strip_rows(height: int, world: int, rank: int, r: int) -> dict:
    """Rows of rank `rank`: owned [lo, hi), held [lo - top, hi + bottom) with
    top/bottom the halo rows present (clipped at the image edges)."""
    if not (0 <= rank < world) or height < world:
        raise ValueError("need 0 <= rank < world <= height")
    base, extra = divmod(height, world)
    if world > 1 and base < r:
        # a halo then reaches past the neighbouring strip: not supported
        raise ValueError(f"strips of {base} rows are thinner than the window radius {r}")
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    top = min(r, lo)
    bottom = min(r, height - hi)
    return {"lo": lo, "hi": hi, "top": top, "bottom": bottom, "held": (lo - top, hi + bottom)}


def halo_exchange(local, height: int, world: int, rank: int, r: int, dist) -> None:
    """Fill the halo rows of `local` ([planes][held rows][width], the new
    frame's records) from the neighbouring ranks' owned rows, in place."""
    s = strip_rows(height, world, rank, r)
    own0 = s["top"]                      # first owned row inside `local`
    own1 = own0 + (s["hi"] - s["lo"])    # one past the last owned row
    ops = []
    if rank > 0:
        # my first owned rows fill the bottom halo of the rank above (r rows:
        # strips are at least r rows thick); its last rows fill my top halo
        send_up = local[:, own0:own0 + min(r, height - s["lo"])].contiguous()
        recv_top = local.new_empty(local[:, 0:s["top"]].shape)
        ops.append(dist.P2POp(dist.isend, send_up, rank - 1))
        ops.append(dist.P2POp(dist.irecv, recv_top, rank - 1))
    if rank < world - 1:
        send_down = local[:, own1 - min(r, s["hi"]):own1].contiguous()
        recv_bottom = local.new_empty(local[:, own1:own1 + s["bottom"]].shape)
        ops.append(dist.P2POp(dist.isend, send_down, rank + 1))
        ops.append(dist.P2POp(dist.irecv, recv_bottom, rank + 1))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    if rank > 0:
        local[:, 0:s["top"]] = recv_top
    if rank < world - 1:
        local[:, own1:own1 + s["bottom"]] = recv_bottom


def merge_events(per_rank: list, row_offsets: list):
    """Concatenate per-rank event arrays (structured, fields frame/x/y/polarity,
    y relative to the rank's first owned row) into the whole image's list in
    canonical (frame, row, column, repeat) order."""
    import numpy as np
    parts = []
    for ev, off in zip(per_rank, row_offsets):
        e = ev.copy()
        e["y"] = e["y"] + off
        parts.append(e)
    if not parts:
        return np.zeros(0)
    allev = np.concatenate(parts)
    # frame-major: rank order already gives row order within a frame
    order = np.argsort(allev["frame"], kind="stable")
    return allev[order]


def held_frame(frame: dict, rows: dict) -> dict:
    """The held rows [lo - top, hi + bottom) of a whole frame's planes
    ([C][H][W] or [H][W] tensors), each made contiguous."""
    a, b = rows["held"]
    return {k: v[..., a:b, :].contiguous() for k, v in frame.items() if v is not None}


class StripSimulator:
    """Rank `rank` of `world` in the strip split of one sequence of cfg.height
    rows: a Simulator over the held rows, reporting the owned rows.

    push() takes the held rows of a frame (held_frame() cuts them out of a
    whole frame; a multi-GPU run assembles them from its own rows and the halo
    exchange).  events() returns the owned rows' events with y relative to the
    first owned row (merge_events() with offsets lo joins the ranks);
    denoised() the owned rows of alpha and of the flags."""

    def __init__(self, cfg, world: int, rank: int, stream=None):
        from dataclasses import replace
        from . import Simulator
        self.rows = strip_rows(cfg.height, world, rank, cfg.radius)
        a, b = self.rows["held"]
        self.cfg = replace(cfg, height=b - a)
        self.sim = Simulator(self.cfg, stream)
        self._own = (self.rows["top"], self.rows["top"] + self.rows["hi"] - self.rows["lo"])

    def close(self):
        self.sim.close()

    def push(self, held: dict) -> None:
        self.sim.push(held)

    def events(self):
        ev = self.sim.events()
        r0, r1 = self._own
        keep = (ev["y"] >= r0) & (ev["y"] < r1)
        out = ev[keep]
        out["y"] = out["y"] - r0
        return out

    def denoised(self):
        alpha, flags = self.sim.denoised()
        r0, r1 = self._own
        return alpha[r0:r1], flags[r0:r1]

    def set_state(self, l_last, beta, xc) -> None:
        """Per-pixel model of the held rows from whole-image arrays
        ([H*W], [H*W][7], [H*W][7], as Simulator.get_state returns them)."""
        a, b = self.rows["held"]
        W = self.cfg.width
        self.sim.set_state(l_last[a * W:b * W], beta[a * W:b * W], xc[a * W:b * W])
