"""Analytic box scene for the Monte Carlo renderer: an open-fronted room with
coloured diffuse walls, a checkered back wall, a rectangular area light in the
ceiling and moving diffuse spheres.  Numbers only: the renderer and its
oracle read this description, neither shares code through it."""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class Sphere:
    center: tuple           # at frame 0
    velocity: tuple         # added per frame
    radius: float
    albedo: tuple


@dataclass
class RenderScene:
    width: int = 160
    height: int = 120
    spp: int = 4
    max_bounces: int = 2    # surface interactions per path (1: direct light only)
    seed: int = 0
    cam_pos: tuple = (0.0, 0.0, 1.4)    # inside the room, the open front behind it
    tan_half_fov_y: float = 0.41421356   # 45 degree vertical field of view
    box: tuple = (1.0, 1.0, 1.5)         # half extents; the room's front (z = +box[2]) is open
    wall_albedo: tuple = ((0.63, 0.065, 0.05), (0.14, 0.45, 0.091), (0.725, 0.71, 0.68),
                          (0.725, 0.71, 0.68), (0.725, 0.71, 0.68))   # left, right, floor, ceiling, back
    back_albedo2: tuple = (0.2, 0.2, 0.25)
    checker: float = 0.25
    light: tuple = (-0.3, 0.3, -0.6, 0.0)   # x0, x1, z0, z1 on the ceiling
    light_radiance: tuple = (17.0, 12.0, 4.0)
    eps: float = 1e-4
    spheres: list = field(default_factory=list)


def cornell(width: int = 160, height: int = 120, spp: int = 4, seed: int = 0, max_bounces: int = 2) -> RenderScene:
    """The default box with three spheres moving through it."""
    return RenderScene(width=width, height=height, spp=spp, seed=seed, max_bounces=max_bounces, spheres=[
        Sphere((-0.45, -0.65, -0.6), (0.012, 0.0, 0.004), 0.35, (0.8, 0.8, 0.8)),
        Sphere((0.45, -0.7, 0.1), (-0.008, 0.0, -0.006), 0.3, (0.2, 0.4, 0.8)),
        Sphere((0.0, 0.2, -0.9), (0.0, -0.01, 0.0), 0.2, (0.9, 0.6, 0.1)),
    ])
