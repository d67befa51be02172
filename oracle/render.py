"""CPU oracle of the Monte Carlo test-scene renderer.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

The renderer's output is decided by floating-point comparisons (which wall or
sphere a ray reaches, whether a shadow ray is blocked), so this restatement
takes every decision in the renderer's own precision: numpy float32 with one
rounding per operation, in the order the estimator is written down below,
which makes the comparison with the CUDA renderer exact.  Random numbers
come from the Philox4x32-10 definition in ``scenes/philox.py``.

Estimator (per pixel, samples s = 0..spp-1): camera ray through the pixel
jittered by (u0, u1) of Philox call 1; at interaction b: nearest of the room's
walls (open front: the path ends) and the spheres beyond eps; camera rays that
reach the ceiling light add its radiance and end; otherwise next-event
estimation to the light point (x0 + u0 (x1 - x0), box_y, z0 + u1 (z1 - z0)) of
call 2b + 2 with G = cos_s cos_l area / (pi d^2), unless a sphere lies between;
then (if interactions remain) a cosine-weighted direction from (u2, u3) with
the orthonormal basis of Duff et al. (2017).  cos/sin(2 pi u) come from the
Taylor polynomials of sin and cos after a quarter-turn reduction.
"""
from __future__ import annotations

import numpy as np
import torch

from scenes.philox import philox4x32

f32 = np.float32
INF = f32(np.inf)


def _unit(w) -> np.ndarray:
    return (np.asarray(w, np.uint32) >> 8).astype(f32) * f32(5.9604644775390625e-8)


def _philox(pix, smp, call, seed, frame):
    c0 = torch.from_numpy(pix.astype(np.int64))
    c1 = torch.full_like(c0, int(smp))
    c2 = torch.full_like(c0, int(call))
    c3 = torch.zeros_like(c0)
    out = philox4x32(c0, c1, c2, c3, int(seed), int(frame))
    return [o.numpy().astype(np.uint32) for o in out]


def _dot(a, b):
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]


def _sincos_turns(u):
    u4 = u * f32(4.0)
    qf = np.floor(u4)
    q = qf.astype(np.int64)
    th = (u4 - qf) * f32(1.57079637)
    t2 = th * th
    ps = np.full_like(th, f32(-2.50521084e-8))
    for k in (2.75573188e-6, -1.98412701e-4, 8.33333377e-3, -1.66666672e-1, 1.0):
        ps = ps * t2 + f32(k)
    sn = ps * th
    pc = np.full_like(th, f32(2.08767570e-9))
    for k in (-2.75573188e-7, 2.48015876e-5, -1.38888892e-3, 4.16666679e-2, -0.5):
        pc = pc * t2 + f32(k)
    cs = pc * t2 + f32(1.0)
    c = np.select([q == 0, q == 1, q == 2], [cs, -sn, -cs], sn)
    s = np.select([q == 0, q == 1, q == 2], [sn, cs, -sn], -cs)
    return c.astype(f32), s.astype(f32)


def _cosine_direction(n, uz, uphi):
    """Cosine-weighted direction about the unit normal n (three float32 arrays)
    from two uniform numbers: sin^2 of the polar angle uz, azimuth 2 pi uphi,
    in the orthonormal basis of Duff et al. (2017)."""
    cph, sph = _sincos_turns(uphi)
    rr = np.sqrt(uz)
    lz = np.sqrt(np.maximum(f32(1.0) - uz, f32(0.0)))
    lx, ly = rr * cph, rr * sph
    sg = np.where(n[2] >= 0, f32(1.0), f32(-1.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        aa = f32(-1.0) / (sg + n[2])
    bb = (n[0] * n[1]) * aa
    t1 = [f32(1.0) + (sg * (n[0] * n[0])) * aa, sg * bb, -(sg * n[0])]
    t2 = [bb, sg + (n[1] * n[1]) * aa, -n[1]]
    return [(t1[i] * lx + t2[i] * ly) + n[i] * lz for i in range(3)]


def _hit_spheres(sc, ctr, o, d, eps):
    t_best = np.full(o[0].shape, INF, f32)
    kind = np.full(o[0].shape, -1, np.int64)
    for j, sp in enumerate(sc.spheres):
        oc = [o[i] - ctr[j][i] for i in range(3)]
        b = _dot(oc, d)
        r = f32(sp.radius)
        cc = _dot(oc, oc) - r * r
        disc = b * b - cc
        ok = disc > 0
        sq = np.sqrt(np.where(ok, disc, f32(0)))
        t = -b - sq
        t = np.where(t > eps, t, -b + sq)
        take = ok & (t > eps) & (t < t_best)
        t_best = np.where(take, t, t_best)
        kind = np.where(take, 8 + j, kind)
    return t_best, kind


def _hit_walls(sc, o, d):
    bx, by, bz = (f32(v) for v in sc.box)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.full(o[0].shape, INF, f32)
        kind = np.full(o[0].shape, 5, np.int64)
        tx_p = (bx - o[0]) / d[0]
        tx_n = (-bx - o[0]) / d[0]
        t = np.where(d[0] > 0, tx_p, np.where(d[0] < 0, tx_n, t))
        kind = np.where(d[0] > 0, 1, np.where(d[0] < 0, 0, kind))
        ty = np.where(d[1] > 0, (by - o[1]) / d[1], (-by - o[1]) / d[1])
        ky = np.where(d[1] > 0, 3, 2)
        take = (d[1] != 0) & (ty < t)
        t, kind = np.where(take, ty, t), np.where(take, ky, kind)
        tz = np.where(d[2] < 0, (-bz - o[2]) / d[2], (bz - o[2]) / d[2])
        kz = np.where(d[2] < 0, 4, 5)
        take = (d[2] != 0) & (tz < t)
        t, kind = np.where(take, tz, t), np.where(take, kz, kind)
    return t.astype(f32), kind


def render(sc, frame: int) -> dict:
    """All outputs of one frame as float32 arrays (radiance [3][H][W], variance
    [H][W], normal [3][H][W], albedo [3][H][W], depth [H][W])."""
    W, H = sc.width, sc.height
    n_pix = W * H
    pix = np.arange(n_pix, dtype=np.int64)
    px = (pix % W).astype(f32)
    py = (pix // W).astype(f32)
    tf = f32(frame)
    ctr = [[f32(sp.center[i]) + tf * f32(sp.velocity[i]) for i in range(3)] for sp in sc.spheres]
    tany = f32(sc.tan_half_fov_y)
    tanx = (tany * f32(W)) / f32(H)
    L0, L1, L2, L3 = (f32(v) for v in sc.light)
    lw, lh = L1 - L0, L3 - L2
    area = lw * lh
    eps = f32(sc.eps)
    Le = [f32(v) for v in sc.light_radiance]
    walls = [[f32(c) for c in a] for a in sc.wall_albedo]
    alb2 = [f32(c) for c in sc.back_albedo2]
    chk = f32(sc.checker)
    nwx = [1, -1, 0, 0, 0]
    nwy = [0, 0, 1, -1, 0]
    nwz = [0, 0, 0, 0, 1]
    zeros = lambda: np.zeros(n_pix, f32)
    acc = [zeros() for _ in range(3)]
    sy, sy2 = zeros(), zeros()
    fn = [zeros() for _ in range(3)]
    fal = [zeros() for _ in range(3)]
    fdp = zeros()
    for smp in range(sc.spp):
        jit = _philox(pix, smp, 1, sc.seed, frame)
        sxp = (((px + _unit(jit[0])) / f32(W)) * f32(2.0) - f32(1.0)) * tanx
        syp = (f32(1.0) - ((py + _unit(jit[1])) / f32(H)) * f32(2.0)) * tany
        inv = f32(1.0) / np.sqrt((sxp * sxp + syp * syp) + f32(1.0))
        o = [np.full(n_pix, f32(c), f32) for c in sc.cam_pos]
        d = [sxp * inv, syp * inv, -inv]
        thr = [np.ones(n_pix, f32) for _ in range(3)]
        L = [zeros() for _ in range(3)]
        alive = np.ones(n_pix, bool)
        for b in range(sc.max_bounces):
            tw, kw = _hit_walls(sc, o, d)
            ts, ks = _hit_spheres(sc, ctr, o, d, eps)
            use_s = ts < tw
            t = np.where(use_s, ts, tw)
            kind = np.where(use_s, ks, kw)
            alive &= kind != 5
            tt = np.where(alive, t, f32(0))
            x = [o[i] + tt * d[i] for i in range(3)]
            # surface normal and albedo
            n = [zeros(), zeros(), zeros()]
            a = [zeros(), zeros(), zeros()]
            for k in range(5):
                m = kind == k
                n[0] = np.where(m, f32(nwx[k]), n[0])
                n[1] = np.where(m, f32(nwy[k]), n[1])
                n[2] = np.where(m, f32(nwz[k]), n[2])
                for c in range(3):
                    a[c] = np.where(m, walls[k][c], a[c])
            if chk > 0:
                with np.errstate(invalid="ignore"):
                    ix = np.floor(x[0] / chk).astype(np.int64)
                    iy = np.floor(x[1] / chk).astype(np.int64)
                odd = (kind == 4) & (((ix + iy) & 1) == 1)
                for c in range(3):
                    a[c] = np.where(odd, alb2[c], a[c])
            for j, sp in enumerate(sc.spheres):
                m = kind == 8 + j
                inv_r = f32(1.0) / f32(sp.radius)
                for i in range(3):
                    n[i] = np.where(m, (x[i] - ctr[j][i]) * inv_r, n[i])
                for c in range(3):
                    a[c] = np.where(m, f32(sp.albedo[c]), a[c])
            light = (kind == 3) & (x[0] >= L0) & (x[0] <= L1) & (x[2] >= L2) & (x[2] <= L3)
            if b == 0:
                for i in range(3):
                    fn[i] = fn[i] + np.where(alive, n[i], f32(0))
                    fal[i] = fal[i] + np.where(alive, a[i], f32(0))
                fdp = fdp + np.where(alive, tt, f32(0))
                for c in range(3):
                    L[c] = np.where(alive & light, L[c] + Le[c], L[c])
            alive &= ~light
            r = _philox(pix, smp, 2 * b + 2, sc.seed, frame)
            lp = [L0 + _unit(r[0]) * lw, np.full(n_pix, f32(sc.box[1]), f32), L2 + _unit(r[1]) * lh]
            w = [lp[i] - x[i] for i in range(3)]
            d2 = _dot(w, w)
            dist = np.sqrt(d2)
            winv = f32(1.0) / dist
            wl = [w[i] * winv for i in range(3)]
            cs = _dot(n, wl)
            cl = wl[1]
            sh_t, _ = _hit_spheres(sc, ctr, x, wl, eps)
            lit = alive & (cs > 0) & (cl > 0) & ~(sh_t < dist - eps)
            g = ((cs * cl) * area) / (f32(3.14159274) * d2)
            for c in range(3):
                L[c] = np.where(lit, L[c] + ((thr[c] * a[c]) * Le[c]) * g, L[c])
            if b + 1 >= sc.max_bounces:
                break
            d = _cosine_direction(n, _unit(r[2]), _unit(r[3]))
            o = x
            thr = [thr[c] * a[c] for c in range(3)]
            if not alive.any():
                break
        for c in range(3):
            acc[c] = acc[c] + L[c]
        Y = (f32(0.2126) * L[0] + f32(0.7152) * L[1]) + f32(0.0722) * L[2]
        sy = sy + Y
        sy2 = sy2 + Y * Y
    nf = f32(sc.spp)
    out = {"radiance": np.stack([acc[c] / nf for c in range(3)]),
           "normal": np.stack([fn[i] / nf for i in range(3)]),
           "albedo": np.stack([fal[c] / nf for c in range(3)]),
           "depth": fdp / nf}
    if sc.spp > 1:
        var = np.maximum((sy2 - (sy * sy) / nf) / (nf * (nf - f32(1.0))), f32(0.0))
    else:
        var = zeros()
    out["variance"] = var
    return {k: v.reshape((-1, H, W)) if v.ndim == 2 else v.reshape(H, W) for k, v in out.items()}
