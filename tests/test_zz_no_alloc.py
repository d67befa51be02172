"""The allocation-free event writer, checked against the simulator context.

esim_ad_write_events_noalloc is for callers that cannot call cudaMalloc where
they need events written (allocation-free stream capture, latency-critical
loops, plugins whose host framework owns all device memory).  It keeps its
scratch in a fixed array inside the library.  Here a context runs a short
sequence; each frame's events, turned back into a signed per-pixel count map,
go through the allocation-free call, and the records must equal the
context's own, exactly (integer work).  Two calls in a row check that the
shared array is cleared between calls.  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _count_map(ev, H, W):
    m = np.zeros((H, W), np.int32)
    np.add.at(m, (ev["y"].astype(np.int64), ev["x"].astype(np.int64)), ev["polarity"].astype(np.int32))
    return m


def test_noalloc_writer_matches_context_events_two_calls():
    import torch
    import paper_2303_02608_gb300 as m
    from paper_2303_02608_gb300 import EVENT_DTYPE, SimConfig, Simulator
    from scenes import Scene, SceneConfig

    H, W = 72, 100
    cfg = SceneConfig(kind="rects", width=W, height=H, frames=5, spp=4, seed=21, rgb=True, n_rects=10,
                      bg_depth=10.0)
    frames = Scene(cfg).sequence()
    sim = Simulator(SimConfig(width=W, height=H, radius=3, frames=2, contrast=0.15,
                              mode=m.ESIM_AD_EXHAUSTIVE))
    per_frame = []
    for fr in frames:
        sim.push({k: fr[k].cuda() for k in ("radiance", "normal", "albedo", "depth")})
        per_frame.append(sim.events())
    sim.close()
    calls = [(t, per_frame[t]) for t in (3, 4)]
    assert all(len(ev) > 0 for _, ev in calls)

    stream = torch.cuda.current_stream()
    for t, ev in calls:                      # two calls in a row share the array
        counts = torch.from_numpy(_count_map(ev, H, W)).cuda()
        cap = len(ev) + 16
        out = torch.zeros(cap * 12, dtype=torch.uint8, device="cuda")
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = m.esim_ad_write_events_noalloc(counts.data_ptr(), W, H, t, out.data_ptr(), cap,
                                            total.data_ptr(), stream.cuda_stream)
        assert st == m.ESIM_AD_OK
        torch.cuda.synchronize()
        n = int(total.item())
        assert n == len(ev)
        got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=EVENT_DTYPE)[:n]
        assert np.array_equal(got[["frame", "x", "y", "polarity"]], ev[["frame", "x", "y", "polarity"]])

    # sizes beyond the fixed scratch are refused before any GPU work
    big = m.esim_ad_write_events_noalloc(counts.data_ptr(), 65535, 65535, 0, out.data_ptr(), cap,
                                         total.data_ptr(), stream.cuda_stream)
    assert big == m.ESIM_AD_EINVAL
