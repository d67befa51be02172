"""Seeded synthetic stand-ins for the paper's path-traced input frames.

The paper renders its scenes with PBRT-v4 and hands the converter, per frame,
a noisy radiance image plus first-bounce features: normal (3), depth (1) and
texture colour / albedo (3) (Section 3).  Those scenes are not available, so
this module draws frames with the same buffers, shapes and noise structure:

* ``disc``  - a bright disc translating over a horizontal gradient, luminance
  only (the 64x64 smoke workload).
* ``rects`` - moving textured rectangles with piecewise-constant albedo,
  Lambertian shading and painter's-order occlusion, RGB radiance.

Monte Carlo noise at ``spp`` samples per pixel is modelled as a multiplicative
Gamma(k, 1/k) factor (mean 1, variance 1/k), drawn as -(1/k) * sum of k
logarithms of Philox uniforms, independently per pixel, channel and frame.
The per-pixel sample variance the renderer would supply is clean^2 / k,
reduced to luminance with the Rec.709 weights for RGB scenes.

This module is the only code shared by the CUDA path's tests and the oracle's
tests.  It holds none of the method's arithmetic: it only produces inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from .philox import philox4x32, uniform_open01

# Rec.709 luminance weights, used here only to reduce the supplied variance.
_REC709 = (0.2126, 0.7152, 0.0722)
_LIGHT = (0.3, 0.5, 1.0)

_KEY_NOISE = 0x5EED0001
_KEY_LAYOUT = 0x1A70D002
_KEY_BG = 0xB6C0D003


@dataclass
class SceneConfig:
    kind: str = "disc"          # "disc" | "rects"
    width: int = 64
    height: int = 64
    frames: int = 8
    spp: int = 4                # Gamma shape k (integer samples per pixel)
    seed: int = 0
    seq: int = 0                # sequence id, part of every noise counter
    rgb: bool = False           # radiance channels: 1 (luminance) or 3 (RGB)
    n_rects: int = 32
    # disc scene parameters
    disc_radius: float = 12.0
    disc_radiance: float = 2.0
    disc_albedo: float = 0.9
    disc_depth: float = 2.0
    disc_start: tuple = (16.0, 32.0)
    disc_velocity: tuple = (2.0, 0.0)
    bg_depth: float = 5.0
    # textured, panning background (0 = the plain horizontal gradient): square
    # cells of bg_cell pixels with their own RGB albedo, depth and tilted
    # normal, translating by bg_pan pixels per frame (a camera pan)
    bg_cell: int = 0
    bg_pan: tuple = (0.0, 0.0)
    extra: dict = field(default_factory=dict)


# Presets shaped like the workloads the simulator is measured on.
def preset(name: str, **over) -> SceneConfig:
    table = {
        "disc64": dict(kind="disc", width=64, height=64, frames=8, spp=4, seed=0, rgb=False),
        "rects720p": dict(kind="rects", width=1280, height=720, frames=120, spp=4, seed=0,
                          rgb=True, bg_depth=10.0),
        "rects1080p": dict(kind="rects", width=1920, height=1080, frames=240, spp=1, seed=0,
                           rgb=True, bg_depth=10.0),
        "rects512": dict(kind="rects", width=512, height=512, frames=16, spp=2, seed=0,
                         rgb=True, bg_depth=10.0),
        # the same rectangles over a textured background seen by a panning
        # camera: about a tenth to a third of the pixels change features per
        # frame, the density at which the paper regresses (about 28%)
        "pan1080p": dict(kind="rects", width=1920, height=1080, frames=240, spp=1, seed=0,
                         rgb=True, bg_depth=10.0, bg_cell=6, bg_pan=(1.7, 0.7)),
    }
    d = dict(table[name])
    d.update(over)
    return SceneConfig(**d)


def _layout_uniforms(cfg: SceneConfig, n: int) -> list[float]:
    """n layout uniforms in (0,1) for the rectangle scene, keyed by (seed, seq)."""
    blocks = (n + 3) // 4
    idx = torch.arange(blocks, dtype=torch.int64)
    z = torch.zeros_like(idx)
    o = philox4x32(idx, z + 0xFFFF, z + (cfg.seq & 0xFFFFFFFF), z, cfg.seed, _KEY_LAYOUT)
    u = uniform_open01(torch.stack(o, dim=1).reshape(-1))
    return [float(v) for v in u[:n]]


@dataclass
class Rect:
    x0: float
    y0: float
    w: float
    h: float
    vx: float
    vy: float
    depth: float
    normal: tuple
    albedo: list  # [4][4][3]


def rect_layout(cfg: SceneConfig) -> list[Rect]:
    """Draw the rectangles: sides U[H/16, H/4], uniform start, random direction,
    speed U[0.5, 4] px/frame, depth U[1, 10], unit normal with n_z >= 0.7 and a
    4x4 grid of RGB albedo cells U[0.05, 0.95]."""
    per = 10 + 48
    u = _layout_uniforms(cfg, per * cfg.n_rects)
    H, W = cfg.height, cfg.width
    rects = []
    for i in range(cfg.n_rects):
        v = u[i * per:(i + 1) * per]
        w = H / 16 + (H / 4 - H / 16) * v[0]
        h = H / 16 + (H / 4 - H / 16) * v[1]
        x0 = -w / 2 + (W) * v[2]
        y0 = -h / 2 + (H) * v[3]
        ang = 2 * math.pi * v[4]
        spd = 0.5 + 3.5 * v[5]
        depth = 1.0 + 9.0 * v[6]
        nz = 0.7 + 0.3 * v[7]
        phi = 2 * math.pi * v[8]
        s = math.sqrt(max(0.0, 1 - nz * nz))
        normal = (s * math.cos(phi), s * math.sin(phi), nz)
        alb = [[[0.05 + 0.9 * v[10 + (cy * 4 + cx) * 3 + c] for c in range(3)]
                for cx in range(4)] for cy in range(4)]
        rects.append(Rect(x0, y0, w, h, spd * math.cos(ang), spd * math.sin(ang), depth, normal, alb))
    # painter's order: farthest first, nearer rectangles overwrite
    rects.sort(key=lambda r: -r.depth)
    return rects


class Scene:
    """Frame source for one synthetic sequence."""

    def __init__(self, cfg: SceneConfig):
        self.cfg = cfg
        self.rects = rect_layout(cfg) if cfg.kind == "rects" else []

    @property
    def channels(self) -> int:
        return 3 if self.cfg.rgb else 1

    def clean(self, t: int, device="cpu") -> dict:
        """Noise-free buffers of frame t: radiance [C][H][W] and the features."""
        cfg = self.cfg
        H, W = cfg.height, cfg.width
        f64 = torch.float64
        ys = torch.arange(H, dtype=f64, device=device).view(H, 1).expand(H, W) + 0.5
        xs = torch.arange(W, dtype=f64, device=device).view(1, W).expand(H, W) + 0.5
        grad = 0.2 + 0.8 * (xs - 0.5) / max(W - 1, 1)
        normal = torch.zeros(3, H, W, dtype=f64, device=device)
        normal[2] = 1.0
        albedo = grad.unsqueeze(0).repeat(3, 1, 1)
        depth = torch.full((H, W), cfg.bg_depth, dtype=f64, device=device)
        rad = grad.unsqueeze(0).repeat(3, 1, 1)
        if cfg.bg_cell > 0:
            albedo, depth, normal, rad = self._textured_background(t, xs, ys, device)
        if cfg.kind == "disc":
            cx = cfg.disc_start[0] + cfg.disc_velocity[0] * t
            cy = cfg.disc_start[1] + cfg.disc_velocity[1] * t
            m = (xs - cx) ** 2 + (ys - cy) ** 2 <= cfg.disc_radius ** 2
            rad = torch.where(m, torch.full_like(grad, cfg.disc_radiance), grad).unsqueeze(0)
            albedo = torch.where(m.unsqueeze(0), torch.full_like(albedo, cfg.disc_albedo), albedo)
            depth = torch.where(m, torch.full_like(depth, cfg.disc_depth), depth)
            if cfg.rgb:
                rad = rad.repeat(3, 1, 1)
        elif cfg.kind == "rects":
            lx, ly, lz = _LIGHT
            ln = math.sqrt(lx * lx + ly * ly + lz * lz)
            for r in self.rects:
                X = r.x0 + r.vx * t
                Y = r.y0 + r.vy * t
                m = (xs >= X) & (xs < X + r.w) & (ys >= Y) & (ys < Y + r.h)
                if not bool(m.any()):
                    continue
                cxi = torch.clamp(((xs - X) * (4.0 / r.w)).floor().long(), 0, 3)
                cyi = torch.clamp(((ys - Y) * (4.0 / r.h)).floor().long(), 0, 3)
                cell = cyi * 4 + cxi
                alb = torch.tensor(r.albedo, dtype=f64, device=device).reshape(16, 3)
                a = alb[cell].permute(2, 0, 1)                  # [3][H][W]
                ndl = max(0.0, (r.normal[0] * lx + r.normal[1] * ly + r.normal[2] * lz) / ln)
                shade = 0.3 + 0.7 * ndl
                albedo = torch.where(m.unsqueeze(0), a, albedo)
                rad = torch.where(m.unsqueeze(0), a * shade, rad)
                depth = torch.where(m, torch.full_like(depth, r.depth), depth)
                nv = torch.tensor(r.normal, dtype=f64, device=device).view(3, 1, 1).expand(3, H, W)
                normal = torch.where(m.unsqueeze(0), nv, normal)
            if not cfg.rgb:
                rad = (_REC709[0] * rad[0] + _REC709[1] * rad[1] + _REC709[2] * rad[2]).unsqueeze(0)
        else:
            raise ValueError(cfg.kind)
        return {"radiance": rad, "normal": normal, "albedo": albedo, "depth": depth}

    def _textured_background(self, t, xs, ys, device):
        """Background of square cells in world coordinates, seen at an offset of
        bg_pan * t pixels: per cell an RGB albedo U[0.1, 0.9], a depth
        bg_depth * U[0.8, 1.2] and a unit normal tilted by up to ~25 degrees;
        Lambertian shading as for the rectangles."""
        cfg = self.cfg
        f64 = torch.float64
        wx = xs + cfg.bg_pan[0] * t
        wy = ys + cfg.bg_pan[1] * t
        cx = torch.floor(wx / cfg.bg_cell).to(torch.int64)
        cy = torch.floor(wy / cfg.bg_cell).to(torch.int64)
        # counters: cell x, cell y (offset to stay non-negative), sequence
        z = torch.zeros_like(cx)
        w = philox4x32((cx + (1 << 20)) & 0xFFFFFFFF, (cy + (1 << 20)) & 0xFFFFFFFF,
                       z + (cfg.seq & 0xFFFFFFFF), z, cfg.seed, _KEY_BG)
        w2 = philox4x32((cx + (1 << 20)) & 0xFFFFFFFF, (cy + (1 << 20)) & 0xFFFFFFFF,
                        z + (cfg.seq & 0xFFFFFFFF), z + 1, cfg.seed, _KEY_BG)
        u = [uniform_open01(v) for v in w] + [uniform_open01(v) for v in w2]
        albedo = torch.stack([0.1 + 0.8 * u[0], 0.1 + 0.8 * u[1], 0.1 + 0.8 * u[2]], 0)
        depth = cfg.bg_depth * (0.8 + 0.4 * u[3])
        tx, ty = 0.45 * (u[4] - 0.5) * 2, 0.45 * (u[5] - 0.5) * 2
        n = torch.stack([tx, ty, torch.ones_like(tx)], 0)
        n = n / torch.sqrt((n * n).sum(0, keepdim=True))
        lx, ly, lz = _LIGHT
        ln = math.sqrt(lx * lx + ly * ly + lz * lz)
        ndl = torch.clamp((n[0] * lx + n[1] * ly + n[2] * lz) / ln, min=0.0)
        rad = albedo * (0.3 + 0.7 * ndl).unsqueeze(0)
        return albedo.to(f64), depth.to(f64), n.to(f64), rad.to(f64)

    def gamma_factor(self, t: int, device="cpu") -> torch.Tensor:
        """Multiplicative Gamma(k, 1/k) noise, shape [C][H][W], float64."""
        cfg = self.cfg
        C, H, W = self.channels, cfg.height, cfg.width
        k = int(cfg.spp)
        n = H * W
        pix = torch.arange(n, dtype=torch.int64, device=device)
        z = torch.zeros_like(pix)
        acc = torch.zeros(C, n, dtype=torch.float64, device=device)
        for ch in range(C):
            for b in range((k + 3) // 4):
                words = philox4x32(pix, z + (t & 0xFFFFFFFF), z + ((cfg.seq << 8) | ch) % (1 << 32),
                                   z + b, cfg.seed, _KEY_NOISE)
                for j in range(4):
                    if 4 * b + j < k:
                        acc[ch] -= torch.log(uniform_open01(words[j]))
        return (acc / k).view(C, H, W)

    def frame(self, t: int, device="cpu") -> dict:
        """Noisy frame t as float32 tensors: radiance [C][H][W], variance [H][W],
        normal [3][H][W], albedo [3][H][W], depth [H][W], clean [C][H][W]."""
        c = self.clean(t, device)
        g = self.gamma_factor(t, device)
        clean = c["radiance"]
        noisy = clean * g
        k = float(self.cfg.spp)
        if clean.shape[0] == 3:
            var = sum((_REC709[i] ** 2) * clean[i] ** 2 for i in range(3)) / k
        else:
            var = clean[0] ** 2 / k
        f32 = torch.float32
        return {
            "radiance": noisy.to(f32).contiguous(),
            "variance": var.to(f32).contiguous(),
            "normal": c["normal"].to(f32).contiguous(),
            "albedo": c["albedo"].to(f32).contiguous(),
            "depth": c["depth"].to(f32).contiguous(),
            "clean": clean.to(f32).contiguous(),
        }

    def sequence(self, frames: int | None = None, device="cpu") -> list[dict]:
        n = self.cfg.frames if frames is None else frames
        return [self.frame(t, device) for t in range(n)]


def batch_configs(n_seq: int = 48, seed: int = 0) -> list[SceneConfig]:
    """Configs of the batched workload: resolution from {256^2, 640x480, 1280x720,
    1920x1080}, 32-128 frames, 2-16 spp, drawn from a seed-keyed meta stream;
    sequence i uses scene seed 1000 + i."""
    res = [(256, 256), (640, 480), (1280, 720), (1920, 1080)]
    idx = torch.arange(n_seq, dtype=torch.int64)
    z = torch.zeros_like(idx)
    o = philox4x32(idx, z + 0xBA7C, z, z, seed, _KEY_LAYOUT)
    u = [uniform_open01(w) for w in o]
    out = []
    for i in range(n_seq):
        w, h = res[min(3, int(float(u[0][i]) * 4))]
        frames = 32 + min(96, int(float(u[1][i]) * 97))
        spp = 2 + min(14, int(float(u[2][i]) * 15))
        out.append(SceneConfig(kind="rects", width=w, height=h, frames=frames, spp=spp,
                               seed=1000 + i, seq=i, rgb=True, bg_depth=10.0))
    return out
