"""The allocation-free event writer, checked against the simulator context.

esim_ad_write_events_noalloc is for callers that cannot call cudaMalloc where
they need events written (latency-critical loops that cannot take
cudaMalloc's implicit device synchronisation, plugins whose host framework
owns all device memory).  It keeps its scratch in a fixed array inside the
library.  Here a context runs a short sequence; each frame's events, turned
back into a signed per-pixel count map, go through the allocation-free call,
and the records must equal the context's own, exactly (integer work).  Two
calls in a row check that the shared array is cleared between calls, and the
device memory held by torch and free on the device is the same before and
after the calls.  This file sorts last so that a run stopping at the first
failure has already run every other test.
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
    torch.cuda.synchronize()
    held0 = torch.cuda.memory_allocated()
    outs = []
    for t, ev in calls:   # inputs and outputs allocated before the calls
        cap = len(ev) + 16
        outs.append((t, ev, torch.from_numpy(_count_map(ev, H, W)).cuda(),
                     torch.zeros(cap * 12, dtype=torch.uint8, device="cuda"), cap,
                     torch.zeros(1, dtype=torch.int64, device="cuda")))
    torch.cuda.synchronize()
    held1 = torch.cuda.memory_allocated()
    free1 = torch.cuda.mem_get_info()[0]
    for t, ev, counts, out, cap, total in outs:   # two calls in a row share the array
        st = m.esim_ad_write_events_noalloc(counts.data_ptr(), W, H, t, out.data_ptr(), cap,
                                            total.data_ptr(), stream.cuda_stream)
        assert st == m.ESIM_AD_OK
        torch.cuda.synchronize()
        n = int(total.item())
        assert n == len(ev)
        got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=EVENT_DTYPE)[:n]
        assert np.array_equal(got[["frame", "x", "y", "polarity"]], ev[["frame", "x", "y", "polarity"]])

    # nothing was allocated by the calls: torch holds what it held, and the
    # device's free memory is unchanged
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == held1 >= held0
    assert torch.cuda.mem_get_info()[0] == free1

    # a count beyond +-2^19 writes nothing and reports UINT64_MAX
    bad = counts.clone()
    bad[0, 0] = 1 << 20
    total.zero_()
    st = m.esim_ad_write_events_noalloc(bad.data_ptr(), W, H, 9, out.data_ptr(), cap, total.data_ptr(),
                                        stream.cuda_stream)
    assert st == m.ESIM_AD_OK
    torch.cuda.synchronize()
    assert int(total.item()) == -1   # UINT64_MAX read as int64

    # sizes beyond the fixed scratch are refused before any GPU work
    big = m.esim_ad_write_events_noalloc(counts.data_ptr(), 65535, 65535, 0, out.data_ptr(), cap,
                                         total.data_ptr(), stream.cuda_stream)
    assert big == m.ESIM_AD_EINVAL
