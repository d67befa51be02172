"""The CUDA renderer against its oracle: every output bit-identical (both
sides take every decision and rounding in IEEE FP32 in the same order), over
image sizes with ragged blocks, sample counts, path lengths, frames and seeds;
then rendered frames driven through the simulator in lock-step with the
simulator's oracle."""
import numpy as np
import pytest
import torch

from oracle import render as R
from scenes.cornell import cornell

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,spp,bounces,frame,seed", [(37, 23, 1, 1, 0, 0), (64, 48, 4, 2, 5, 1),
                                                         (50, 70, 3, 3, 11, 7), (16, 16, 8, 4, 2, 3)])
def test_render_bit_identical(W, H, spp, bounces, frame, seed):
    from paper_2303_02608_gb300 import render
    sc = cornell(width=W, height=H, spp=spp, seed=seed, max_bounces=bounces)
    g = {k: v.cpu().numpy() for k, v in render(sc, frame).items()}
    o = R.render(sc, frame)
    for k in ("radiance", "variance", "normal", "albedo", "depth"):
        assert g[k].shape == o[k].shape
        diff = g[k].view(np.uint32) != o[k].astype(np.float32).view(np.uint32)
        assert not diff.any(), f"{k}: {int(diff.sum())} values differ (first at {np.argwhere(diff)[0]})"


def test_rendered_sequence_through_simulator():
    """Rendered noisy frames (4 spp) -> adaptive simulator, lock-step with the
    FP64 oracle on the same frames (with the variance guard, which reads the
    renderer's variance plane)."""
    from lockstep import run
    from oracle import Oracle, OracleConfig
    from paper_2303_02608_gb300 import SimConfig, Simulator, render
    sc = cornell(width=80, height=60, spp=4, max_bounces=2)
    frames = []
    for t in range(6):
        f = render(sc, t)
        frames.append({k: v.cpu() for k, v in f.items()})
    for kappa in (0.0, 3.0):
        sim = Simulator(SimConfig(width=80, height=60, radius=3, frames=3, contrast=0.2, rgb=True, guard_kappa=kappa))
        orc = Oracle(OracleConfig(80, 60, radius=3, frames=3, channels=3, contrast=0.2, guard_kappa=kappa))
        rep = run(frames, sim, orc, 0.2)
        sim.close()
        assert rep["regressed"] > 0 and rep["events"] > 0


def test_render_empty_room_and_wide_view():
    """No spheres, plain back wall, a view that takes in the light: still bit-identical."""
    from paper_2303_02608_gb300 import render
    sc = cornell(width=24, height=40, spp=2, seed=9, max_bounces=3)
    sc.spheres = []
    sc.checker = 0.0
    sc.tan_half_fov_y = 0.9
    g = {k: v.cpu().numpy() for k, v in render(sc, 4).items()}
    o = R.render(sc, 4)
    for k in g:
        assert np.array_equal(g[k].view(np.uint32), o[k].astype(np.float32).view(np.uint32)), k


# Physics pins on the CUDA renderer's own output (the same facts the oracle is
# pinned to, checked here without the oracle): the radiance of a directly seen
# emitter, the point-light limit of direct lighting on the floor, exact
# linearity in the light's radiance, and light added by a second interaction.

def _np(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_gpu_directly_seen_light_is_exact():
    from paper_2303_02608_gb300 import render
    sc = cornell(width=64, height=48, spp=4)
    sc.tan_half_fov_y = 0.9          # wide enough to see the ceiling light
    out = _np(render(sc, 0))
    seen = np.all(out["radiance"] == np.array(sc.light_radiance, np.float32)[:, None, None], axis=0)
    assert seen.sum() > 10
    assert np.all(out["variance"][seen] == 0)
    assert np.all(out["normal"][1][seen] == -1) and np.all(out["depth"][seen] > 0)


def test_gpu_floor_matches_point_light_limit():
    """A 1 cm x 1 cm light at the ceiling centre, direct light only: the floor
    radiance tends to rho Le A cos_s cos_l / (pi d^2) at the floor point each
    pixel's centre ray reaches."""
    from paper_2303_02608_gb300 import render
    from scenes.cornell import RenderScene
    sc = RenderScene(width=96, height=96, spp=16, max_bounces=1, checker=0.0, spheres=[],
                     light=(-0.005, 0.005, -0.005, 0.005), light_radiance=(1000.0, 1000.0, 1000.0),
                     tan_half_fov_y=0.6, cam_pos=(0.0, 0.0, 1.4))
    out = _np(render(sc, 0))
    W, H = sc.width, sc.height
    ys, xs = np.mgrid[0:H, 0:W]
    tanx = sc.tan_half_fov_y * W / H
    sx = ((xs + 0.5) / W * 2 - 1) * tanx
    sy = (1 - (ys + 0.5) / H * 2) * sc.tan_half_fov_y
    d = np.stack([sx, sy, -np.ones_like(sx)]) / np.sqrt(sx ** 2 + sy ** 2 + 1)
    t = (-sc.box[1] - sc.cam_pos[1]) / np.where(d[1] < 0, d[1], np.nan)
    p = np.stack([sc.cam_pos[i] + t * d[i] for i in range(3)])
    on_floor = (d[1] < 0) & (np.abs(p[0]) < 0.9) & (p[2] > -1.4) & (p[2] < 1.3) & (out["normal"][1] == 1)
    w = np.stack([-p[0], sc.box[1] - p[1], -p[2]])
    d2 = (w ** 2).sum(0)
    cos = w[1] / np.sqrt(d2)
    expect = np.array(sc.wall_albedo[2])[:, None, None] * 1000.0 * 1e-4 * cos ** 2 / (np.pi * d2)
    rel = np.abs(out["radiance"][:, on_floor] - expect[:, on_floor]) / expect[:, on_floor]
    assert on_floor.sum() > 500
    assert np.median(rel) < 0.01 and rel.max() < 0.06


def test_gpu_linear_in_light_radiance():
    from paper_2303_02608_gb300 import render
    sc = cornell(width=40, height=30, spp=2)
    a = _np(render(sc, 3))["radiance"]
    sc.light_radiance = tuple(2 * v for v in sc.light_radiance)
    b = _np(render(sc, 3))["radiance"]
    assert np.array_equal(b, 2 * a)


def test_gpu_second_interaction_only_adds_light():
    from paper_2303_02608_gb300 import render
    r1 = _np(render(cornell(width=40, height=30, spp=2, max_bounces=1), 2))["radiance"]
    r2 = _np(render(cornell(width=40, height=30, spp=2, max_bounces=2), 2))["radiance"]
    assert np.all(r2 >= r1) and (r2 > r1).mean() > 0.5
