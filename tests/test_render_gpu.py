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
