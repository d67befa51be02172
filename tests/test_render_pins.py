"""Pins of the renderer oracle (oracle/render.py) against facts outside
itself: the library sine and cosine, the radiance of a directly seen emitter,
the point-light limit of the direct-lighting integral on the floor, exact
linearity in the light's radiance, and the ordering of one- and two-interaction
paths that share their random numbers."""
import math

import numpy as np
import pytest

from oracle import render as R
from scenes.cornell import RenderScene, Sphere, cornell


def test_sincos_polynomial_matches_libm():
    u = (np.arange(0, 1 << 16, dtype=np.float64) / (1 << 16)).astype(np.float32)
    c, s = R._sincos_turns(u)
    ref = 2 * np.pi * u.astype(np.float64)
    assert np.abs(c - np.cos(ref)).max() < 3e-7
    assert np.abs(s - np.sin(ref)).max() < 3e-7


def test_directly_seen_light_is_exact():
    sc = cornell(width=64, height=48, spp=4)
    sc.tan_half_fov_y = 0.9          # wide enough to see the ceiling light
    out = R.render(sc, 0)
    rad = out["radiance"]
    seen = np.all(np.isclose(rad, np.array(sc.light_radiance, np.float32)[:, None, None], rtol=0, atol=0), axis=0)
    assert seen.sum() > 10
    assert np.all(out["variance"][seen] == 0)
    # first-hit features of those pixels are the ceiling's
    assert np.all(out["normal"][1][seen] == -1) and np.all(out["depth"][seen] > 0)


def test_floor_matches_point_light_limit():
    """A tiny light (area 1e-4) at the ceiling centre, direct light only: the
    floor radiance tends to rho Le A cos_s cos_l / (pi d^2), evaluated at the
    floor point each pixel's centre ray reaches."""
    sc = RenderScene(width=96, height=96, spp=16, max_bounces=1, checker=0.0, spheres=[],
                     light=(-0.005, 0.005, -0.005, 0.005), light_radiance=(1000.0, 1000.0, 1000.0),
                     tan_half_fov_y=0.6, cam_pos=(0.0, 0.0, 1.4))
    out = R.render(sc, 0)
    W, H = sc.width, sc.height
    ys, xs = np.mgrid[0:H, 0:W]
    tanx = sc.tan_half_fov_y * W / H
    sx = ((xs + 0.5) / W * 2 - 1) * tanx
    sy = (1 - (ys + 0.5) / H * 2) * sc.tan_half_fov_y
    d = np.stack([sx, sy, -np.ones_like(sx)]) / np.sqrt(sx ** 2 + sy ** 2 + 1)
    t = (-sc.box[1] - sc.cam_pos[1]) / np.where(d[1] < 0, d[1], np.nan)
    p = np.stack([sc.cam_pos[i] + t * d[i] for i in range(3)])
    on_floor = (d[1] < 0) & (np.abs(p[0]) < 0.9) & (p[2] > -1.4) & (p[2] < 1.3) & (out["normal"][1] == 1)
    w = np.stack([np.zeros_like(p[0]) - p[0], sc.box[1] - p[1], np.zeros_like(p[0]) - p[2]])
    d2 = (w ** 2).sum(0)
    cos = w[1] / np.sqrt(d2)       # both cosines: floor and light normals are vertical
    A = 0.01 * 0.01
    expect = np.array(sc.wall_albedo[2])[:, None, None] * 1000.0 * A * cos ** 2 / (np.pi * d2)
    rel = np.abs(out["radiance"][:, on_floor] - expect[:, on_floor]) / expect[:, on_floor]
    assert on_floor.sum() > 500
    assert np.median(rel) < 0.01 and rel.max() < 0.06


def test_linear_in_light_radiance():
    sc = cornell(width=40, height=30, spp=2)
    a = R.render(sc, 3)["radiance"]
    sc.light_radiance = tuple(2 * v for v in sc.light_radiance)
    b = R.render(sc, 3)["radiance"]
    assert np.array_equal(b, 2 * a)


def test_second_interaction_only_adds_light():
    sc1 = cornell(width=40, height=30, spp=2, max_bounces=1)
    sc2 = cornell(width=40, height=30, spp=2, max_bounces=2)
    r1, r2 = R.render(sc1, 2)["radiance"], R.render(sc2, 2)["radiance"]
    assert np.all(r2 >= r1) and (r2 > r1).mean() > 0.5


def _scaled_albedos(sc, k):
    import dataclasses
    return dataclasses.replace(
        sc, wall_albedo=tuple(tuple(k * c for c in a) for a in sc.wall_albedo),
        back_albedo2=tuple(k * c for c in sc.back_albedo2),
        spheres=[Sphere(s.center, s.velocity, s.radius, tuple(k * c for c in s.albedo)) for s in sc.spheres])


def test_second_interaction_is_quadratic_in_albedo():
    """Halving every albedo (same geometry, same random numbers) halves the
    light that reaches the camera after one surface interaction and quarters
    what arrives after two: the path throughput carries the first surface's
    albedo into the second interaction's direct light."""
    import dataclasses
    sc = cornell(width=40, height=30, spp=2, max_bounces=2)

    def parts(s):
        one = R.render(dataclasses.replace(s, max_bounces=1), 2)["radiance"].astype(np.float64)
        two = R.render(s, 2)["radiance"].astype(np.float64)
        return one, two - one

    d_full, x_full = parts(sc)
    d_half, x_half = parts(_scaled_albedos(sc, 0.5))
    m = x_full > 1e-3 * x_full.max()
    assert m.mean() > 0.3
    np.testing.assert_allclose(4 * x_half[m], x_full[m], rtol=1e-4)
    seen = d_full == d_half             # the emitter seen directly does not scale
    lit = ~seen & (d_full > 1e-3 * d_full.max())
    assert lit.mean() > 0.3
    np.testing.assert_allclose(2 * d_half[lit], d_full[lit], rtol=1e-5)


def test_variance_of_two_samples():
    """The variance output is the unbiased variance of the pixel mean.  With
    two samples it is (Y0 - Y1)^2 / 4 = (Y0 - mean)^2, where Y0 is the
    one-sample render (sample 0 draws the same random numbers in both) and
    mean the two-sample render, Y the Rec.709 luminance."""
    r1 = R.render(cornell(width=40, height=30, spp=1), 4)
    r2 = R.render(cornell(width=40, height=30, spp=2), 4)
    lum = lambda r: 0.2126 * r[0].astype(np.float64) + 0.7152 * r[1] + 0.0722 * r[2]
    y0, mean = lum(r1["radiance"]), lum(r2["radiance"])
    expect = (y0 - mean) ** 2
    assert (expect > 1e-6 * mean.max() ** 2).mean() > 0.3
    tol = 2e-6 * (mean ** 2 + expect) + 1e-12
    assert np.all(np.abs(r2["variance"] - expect) <= tol)


def test_cosine_weighted_directions():
    """The bounce directions are unit vectors in the normal's hemisphere with
    the moments of the cosine-weighted density p = cos(theta) / pi:
    E[cos theta] = 2/3, E[cos^2 theta] = 1/2, and no mean tangential drift,
    for wall normals (both signs of n_z) and arbitrary sphere normals."""
    rng = np.random.default_rng(5)
    N = 1 << 18
    uz = (rng.integers(0, 1 << 24, N) * 5.9604644775390625e-8).astype(np.float32)
    up = (rng.integers(0, 1 << 24, N) * 5.9604644775390625e-8).astype(np.float32)
    normals = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    v = rng.normal(size=(4, 3))
    normals += [tuple(x / np.linalg.norm(x)) for x in v]
    for nv in normals:
        n = [np.full(N, np.float32(c), np.float32) for c in nv]
        d = np.stack(R._cosine_direction(n, uz, up)).astype(np.float64)
        assert np.abs(np.linalg.norm(d, axis=0) - 1).max() < 1e-5
        c = np.asarray(nv, np.float64) @ d
        assert c.min() > -1e-6
        se = 1 / np.sqrt(N)
        assert abs(c.mean() - 2 / 3) < 5 * se * np.sqrt(1 / 2 - 4 / 9)
        assert abs((c ** 2).mean() - 1 / 2) < 5 * se * np.sqrt(1 / 3 - 1 / 4)
        tang = d - np.outer(np.asarray(nv, np.float64), c)
        assert np.abs(tang.mean(axis=1)).max() < 5 * se
