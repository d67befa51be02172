"""The C-ABI boundary: symbols, struct layout, argument checking, ownership
and error behaviour.  The CPU tests load the library without a GPU; the GPU
tests cover allocation failure, buffer overflow and draining."""
import ctypes
import os
import re
import subprocess
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "esim_ad.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(esim_ad_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_02608_gb300 import build
    build.build()
    import paper_2303_02608_gb300 as m
    return m


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert declared, "no functions parsed from the header"
    assert set(declared) == set(lib.EXPORTS)
    so = lib.load_library()
    for name in declared:
        assert getattr(so, name) is not None


def test_struct_layout_matches_header(lib):
    """sizeof/offsetof from the C compiler equal the ctypes mirrors."""
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "esim_ad.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(esim_ad_config), offsetof(esim_ad_config, contrast),
         offsetof(esim_ad_config, event_capacity), offsetof(esim_ad_config, feature_scale),
         sizeof(esim_ad_frame), offsetof(esim_ad_frame, on_host), offsetof(esim_ad_frame, features),
         offsetof(esim_ad_frame, pitch_elems), sizeof(esim_ad_event), sizeof(esim_ad_stats));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(lib.esim_ad_config), lib.esim_ad_config.contrast.offset,
            lib.esim_ad_config.event_capacity.offset, lib.esim_ad_config.feature_scale.offset,
            ctypes.sizeof(lib.esim_ad_frame), lib.esim_ad_frame.on_host.offset, lib.esim_ad_frame.features.offset,
            lib.esim_ad_frame.pitch_elems.offset, lib.EVENT_DTYPE.itemsize, ctypes.sizeof(lib.esim_ad_stats)]
    assert got == want


def _bad_configs(lib):
    ok = lib.make_config(64, 48)
    yield "struct_size", dict(struct_size=12)
    for k, v in [("width", 0), ("height", -1), ("width", 70000), ("radius", 0), ("radius", 16),
                 ("frames", 0), ("frames", 17), ("mode", 2), ("radiance_fmt", 5), ("contrast", 0.0),
                 ("contrast", float("nan")), ("h", -1.0), ("ridge", 0.0), ("log_eps", -1.0),
                 ("event_capacity", 0), ("feature_fmt", 2), ("precision", 3), ("radiance_fmt", 3)]:
        yield k, {k: v}
    yield "bandwidth", {"bandwidth": 0.0}
    del ok


def test_init_rejects_bad_config_without_touching_gpu(lib):
    so = lib.load_library()
    for name, change in _bad_configs(lib):
        cfg = lib.make_config(64, 48)
        for k, v in change.items():
            if k == "bandwidth":
                cfg.bandwidth[3] = v
            else:
                setattr(cfg, k, v)
        h = ctypes.c_void_p(1234)
        st = so.esim_ad_init(ctypes.byref(cfg), None, ctypes.byref(h))
        assert st == lib.ESIM_AD_EINVAL, name
        assert h.value == 1234, "output pointer must be untouched on error"
    assert so.esim_ad_init(None, None, ctypes.byref(ctypes.c_void_p())) == lib.ESIM_AD_EINVAL
    cfg = lib.make_config(64, 48)
    assert so.esim_ad_init(ctypes.byref(cfg), None, None) == lib.ESIM_AD_EINVAL


def test_null_context_calls(lib):
    so = lib.load_library()
    n = ctypes.c_uint64()
    assert so.esim_ad_push_frame(None, None) == lib.ESIM_AD_EINVAL
    assert so.esim_ad_events(None, None, 0, ctypes.byref(n), 0) == lib.ESIM_AD_EINVAL
    assert so.esim_ad_denoised(None, None, None, 0) == lib.ESIM_AD_EINVAL
    assert so.esim_ad_get_state(None, None, None, None) == lib.ESIM_AD_EINVAL
    assert so.esim_ad_reset(None) == lib.ESIM_AD_EINVAL
    so.esim_ad_destroy(None)
    for code in range(-7, 1):
        assert lib.status_string(code) not in ("unknown status", "")


def test_dense_form_descriptors_checked_on_the_host(lib):
    """Workspace sizes of the differentiation and second-order forms, and their
    rejection of bad descriptors and NULL buffers, need no GPU."""
    so = lib.load_library()
    d = lib.make_wlr_desc(40, 24, 5, radius=3, frames=3)
    assert lib.esim_ad_wlr2_workspace_size(d) == 5 * 2 * 40 * 24 * 16
    assert lib.esim_ad_wlr_workspace_size(d) > 0
    for k, v in (("radius", 0), ("radius", 16), ("frames", 0), ("frames", 17), ("width", 0), ("ridge", 0.0),
                 ("h", -1.0), ("log_eps", -1e-3), ("radiance_fmt", 7), ("struct_size", 4)):
        bad = lib.make_wlr_desc(40, 24, 5)
        setattr(bad, k, v)
        assert lib.esim_ad_wlr2_workspace_size(bad) == 0, k
        assert lib.esim_ad_wlr_workspace_size(bad) == 0, k
    P = ctypes.c_void_p
    assert so.esim_ad_wlr2_forward(ctypes.byref(d), None, P(16), P(16), P(16), P(16), None) == lib.ESIM_AD_EINVAL
    assert so.esim_ad_wlr2_forward(None, P(16), P(16), P(16), P(16), P(16), None) == lib.ESIM_AD_EINVAL
    many = lib.make_wlr_desc(8, 8, 70000)
    assert so.esim_ad_wlr2_forward(ctypes.byref(many), P(16), P(16), P(16), P(16), P(16), None) == \
        lib.ESIM_AD_EINVAL


def test_noalloc_writer_checks_arguments_on_the_host(lib):
    """The allocation-free writer refuses bad arguments before any CUDA call:
    NULL counts or total, NULL events with a capacity, sides outside
    1..65535, and frames above 16,777,216 pixels (the fixed scratch)."""
    f = lib.load_library().esim_ad_write_events_noalloc
    p = 256   # a non-NULL dummy address (never dereferenced: the checks come first)
    EINVAL = lib.ESIM_AD_EINVAL
    assert f(None, 64, 64, 0, p, 10, p, None) == EINVAL          # counts
    assert f(p, 64, 64, 0, p, 10, None, None) == EINVAL          # total_device
    assert f(p, 64, 64, 0, None, 10, p, None) == EINVAL          # events with capacity > 0
    for w, h in ((0, 64), (64, 0), (-1, 64), (65536, 1), (1, 65536)):
        assert f(p, w, h, 0, p, 10, p, None) == EINVAL, (w, h)
    assert f(p, 4097, 4096, 0, p, 10, p, None) == EINVAL         # 16,781,312 pixels
    assert f(p, 65535, 65535, 0, p, 10, p, None) == EINVAL


def test_init_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    so = lib.load_library()
    cfg = lib.make_config(64, 48)
    h = ctypes.c_void_p()
    assert so.esim_ad_init(ctypes.byref(cfg), None, ctypes.byref(h)) == lib.ESIM_AD_ECUDA
    assert h.value is None


def test_product_path_has_no_oracle_dependency():
    """The library package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2303_02608_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower() or f == "__init__.py" and "oracle" not in \
                    re.sub(r'""".*?"""', "", txt, flags=re.S).lower(), f


# ----------------------------------------------------------------- GPU

def _frame(W, H, device="cuda"):
    import torch
    g = torch.Generator().manual_seed(0)
    return {"radiance": torch.rand(3, H, W, generator=g).add_(0.1).to(device),
            "normal": torch.rand(3, H, W, generator=g).to(device),
            "albedo": torch.rand(3, H, W, generator=g).to(device),
            "depth": torch.rand(H, W, generator=g).add_(1).to(device)}


@pytest.mark.gpu
def test_alloc_failure_injection(lib):
    """ESIM_AD_FAULT_ALLOC=k makes the k-th device allocation fail: init returns
    ENOMEM, frees what it had, and the process stays usable."""
    code = (
        "import ctypes, torch, paper_2303_02608_gb300 as m\n"
        "torch.cuda.init()\n"
        "so = m.load_library(); cfg = m.make_config(64, 48); h = ctypes.c_void_p()\n"
        "print(so.esim_ad_init(ctypes.byref(cfg), None, ctypes.byref(h)), h.value)\n")
    for k in (1, 5, 12):
        env = dict(os.environ, ESIM_AD_FAULT_ALLOC=str(k), PYTHONPATH=ROOT)
        out = subprocess.check_output([sys.executable, "-c", code], env=env, cwd=ROOT).decode().split()
        assert int(out[0]) == lib.ESIM_AD_ENOMEM and out[1] == "None"


@pytest.mark.gpu
def test_overflow_is_sticky_and_drain_reports_counts(lib):
    from paper_2303_02608_gb300 import SimConfig, Simulator
    import torch
    W, H = 64, 48
    sim = Simulator(SimConfig(width=W, height=H, radius=2, frames=2, contrast=0.05,
                              mode=lib.ESIM_AD_EXHAUSTIVE, event_capacity=8))
    f0 = _frame(W, H)
    f1 = {k: v.clone() for k, v in f0.items()}
    f1["radiance"] *= 3.0
    sim.push(f0)
    sim.push(f1)
    st, n = lib.esim_ad_events(sim.ctx, 0, 0)
    assert st == lib.ESIM_AD_EOVERFLOW and n > 8
    with pytest.raises(lib.EsimError) as e:
        sim.push(f0)
    assert e.value.status == lib.ESIM_AD_ESTATE
    sim.reset()   # clears the sticky state
    sim.push(f0)
    assert len(sim.events()) == 0
    sim.close()
    torch.cuda.synchronize()


@pytest.mark.gpu
def test_bounded_wait_timeout_is_reported_and_sticky(lib):
    """ESIM_AD_TEST_WITHHOLD_COPY=1 makes every warp of the sparse regression
    kernel skip issuing its first window-box copy and bounds each mbarrier
    wait to 64 polls: the wait on that box gives up with no copy in flight for
    it, the kernel records the timeout and returns.  The host reports
    ETIMEOUT at the next synchronising call, every later call ESTATE, and after
    a reset the context works again (the GPU context was never lost)."""
    from paper_2303_02608_gb300 import SimConfig, Simulator
    import torch
    W, H = 64, 48
    keys = {"ESIM_AD_TEST_WITHHOLD_COPY": "1", "ESIM_AD_SPARSE_MAX": "4294967295"}
    old = {k: os.environ.get(k) for k in keys}
    os.environ.update(keys)
    try:
        sim = Simulator(SimConfig(width=W, height=H, radius=3, frames=2, contrast=0.05,
                                  mode=lib.ESIM_AD_ADAPTIVE))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    f0 = _frame(W, H)
    f1 = {k: v.flip(-1).contiguous() for k, v in f0.items()}   # features move: pixels flag
    sim.push(f0)                    # frame 0 regresses densely (tile-staged kernel)
    sim.push(f1)                    # adaptive frame: the sparse kernel's first copies are withheld
    with pytest.raises(lib.EsimError) as e:
        sim.denoised()
    assert e.value.status == lib.ESIM_AD_ETIMEOUT
    with pytest.raises(lib.EsimError) as e:
        sim.push(f0)
    assert e.value.status == lib.ESIM_AD_ESTATE
    with pytest.raises(lib.EsimError) as e:
        sim.events()
    assert e.value.status == lib.ESIM_AD_ESTATE
    sim.reset()
    sim.push(f0)
    alpha, _ = sim.denoised()
    assert torch.isfinite(alpha).all()
    sim.close()
    torch.cuda.synchronize()


@pytest.mark.gpu
def test_drain_enospace_then_full_drain(lib):
    from paper_2303_02608_gb300 import EVENT_DTYPE, SimConfig, Simulator
    W, H = 40, 24
    sim = Simulator(SimConfig(width=W, height=H, radius=1, frames=1, contrast=0.1,
                              mode=lib.ESIM_AD_EXHAUSTIVE))
    f0 = _frame(W, H)
    f1 = {k: v.clone() for k, v in f0.items()}
    f1["radiance"] *= 2.0
    sim.push(f0)
    sim.push(f1)
    st, n = lib.esim_ad_events(sim.ctx, 0, 0)
    assert st == lib.ESIM_AD_ENOSPACE and n >= W * H * 6  # ln 2 / 0.1 -> 6 crossings each
    small = np.empty(3, EVENT_DTYPE)
    st2, n2 = lib.esim_ad_events(sim.ctx, small.ctypes.data, 3)
    assert st2 == lib.ESIM_AD_ENOSPACE and n2 == n     # nothing drained
    ev = sim.events()
    assert len(ev) == n and np.all(ev["frame"] == 1) and np.all(ev["polarity"] == 1)
    assert len(sim.events()) == 0                      # drained
    st3 = sim.stats()
    assert st3["frames"] == 2 and st3["events"] == n and st3["regressions"] == 2 * W * H
    sim.close()


@pytest.mark.gpu
def test_host_frames_match_device_frames(lib):
    """on_host frames (copied in by the library) give the same events as device frames."""
    from paper_2303_02608_gb300 import SimConfig, Simulator
    from scenes import Scene, SceneConfig
    cfg = SceneConfig(kind="rects", width=96, height=64, frames=5, spp=4, seed=11, rgb=True,
                      n_rects=8, bg_depth=10.0)
    frames = Scene(cfg).sequence()
    outs = []
    for host in (False, True):
        sim = Simulator(SimConfig(width=96, height=64, radius=3, frames=3, contrast=0.15))
        evs = []
        for fr in frames:
            planes = {k: (fr[k].pin_memory() if host else fr[k].cuda())
                      for k in ("radiance", "normal", "albedo", "depth")}
            sim.push(planes)
            evs.append(sim.events())
        outs.append(np.concatenate(evs))
        sim.close()
    assert len(outs[0]) > 0 and np.array_equal(outs[0], outs[1])


@pytest.mark.gpu
def test_pitched_frames_match_dense_frames(lib):
    """Input planes with a row pitch wider than the image (device and pinned
    host frames) give the same alpha, flags and events as densely packed ones;
    a pitch below the width is refused."""
    import torch
    from paper_2303_02608_gb300 import SimConfig, Simulator
    W, H, P = 45, 30, 64
    f0 = _frame(W, H, device="cpu")
    f1 = {k: (v * 1.5 if k == "radiance" else v.flip(-1)).contiguous() for k, v in f0.items()}

    def pitched(f):
        out = {}
        for k, v in f.items():
            w = torch.full(v.shape[:-1] + (P,), -7.0)   # junk beyond the width is never read
            w[..., :W] = v
            out[k] = w.contiguous()
        return out

    results = []
    for mode in ("dense", "pitch_dev", "pitch_host"):
        sim = Simulator(SimConfig(width=W, height=H, radius=3, frames=2, contrast=0.1, mode=lib.ESIM_AD_ADAPTIVE))
        for f in (f0, f1):
            if mode == "dense":
                sim.push({k: v.cuda() for k, v in f.items()})
            elif mode == "pitch_dev":
                sim.push({k: v.cuda() for k, v in pitched(f).items()}, pitch=P)
            else:
                sim.push({k: v.pin_memory() for k, v in pitched(f).items()}, pitch=P)
        a, fl = sim.denoised()
        results.append((a.cpu(), fl.cpu(), sim.events()))
        sim.close()
    for a, fl, ev in results[1:]:
        assert torch.equal(a, results[0][0]) and torch.equal(fl, results[0][1])
        assert np.array_equal(ev, results[0][2])
    sim = Simulator(SimConfig(width=W, height=H, radius=3, frames=2, contrast=0.1))
    with pytest.raises(lib.EsimError) as e:
        sim.push({k: v.cuda() for k, v in f0.items()}, pitch=W - 1)
    assert e.value.status == lib.ESIM_AD_EINVAL
    sim.close()


@pytest.mark.gpu
def test_state_roundtrip_resume(lib):
    """Checkpoint/resume: saving the model mid-sequence into a fresh context and
    continuing gives the same events as an uninterrupted run."""
    from paper_2303_02608_gb300 import SimConfig, Simulator
    from scenes import Scene, SceneConfig
    cfg = SceneConfig(kind="rects", width=80, height=48, frames=6, spp=4, seed=12, rgb=True,
                      n_rects=8, bg_depth=10.0)
    frames = [{k: v.cuda() for k, v in f.items() if k != "clean"} for f in Scene(cfg).sequence()]
    sc = SimConfig(width=80, height=48, radius=2, frames=1, contrast=0.15)
    a = Simulator(sc)
    ev_a = []
    for f in frames:
        a.push(f)
        ev_a.append(a.events())
    b = Simulator(sc)
    for f in frames[:3]:
        b.push(f)
        b.events()
    st = b.get_state()
    c = Simulator(sc)
    c.push(frames[2])   # any frame: the ring (T = 1) and the model are replaced below
    c.events()
    c.set_state(st["l_last"], st["beta"], st["xc"])
    ev_c = []
    for f in frames[3:]:
        c.push(f)
        ev_c.append(c.events())
    got = np.concatenate(ev_c)
    want = np.concatenate(ev_a[3:])
    assert len(want) > 0
    assert np.array_equal(got[["x", "y", "polarity"]], want[["x", "y", "polarity"]])
    for s in (a, b, c):
        s.close()


@pytest.mark.gpu
def test_events_into_pinned_and_device_buffers(lib):
    """events_into drains into the caller's own buffer (pinned host or device)
    with the same records as events(); a buffer too small raises ENOSPACE and
    drains nothing."""
    import torch
    from paper_2303_02608_gb300 import EVENT_DTYPE, SimConfig, Simulator
    W, H = 40, 24
    f0 = _frame(W, H)
    f1 = {k: (v * 2.0 if k == "radiance" else v).contiguous() for k, v in f0.items()}
    runs = []
    for dest in ("events", "pinned", "device"):
        sim = Simulator(SimConfig(width=W, height=H, radius=1, frames=1, contrast=0.1, mode=lib.ESIM_AD_EXHAUSTIVE))
        sim.push(f0)
        sim.push(f1)
        if dest == "events":
            runs.append(sim.events())
        else:
            if dest == "pinned":
                small = torch.empty(12, dtype=torch.uint8, pin_memory=True)
                with pytest.raises(lib.EsimError) as e:
                    sim.events_into(small)
                assert e.value.status == lib.ESIM_AD_ENOSPACE
            buf = torch.empty(1 << 20, dtype=torch.uint8, pin_memory=(dest == "pinned"),
                              device="cuda" if dest == "device" else "cpu")
            n = sim.events_into(buf)
            runs.append(buf.cpu().numpy()[: n * 12].view(EVENT_DTYPE).copy())
        sim.close()
    assert runs[0].size > 0
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2])


def _ring_frames(n):
    """n device frames whose radiance steps up and down, so every frame emits."""
    import torch
    f0 = _frame(40, 24)
    out = []
    for t in range(n):
        s = 1.0 + 0.6 * (t % 3)
        out.append({k: (v * s if k == "radiance" else v).contiguous() for k, v in f0.items()})
    return out


def _ring_sim(lib, capacity):
    from paper_2303_02608_gb300 import SimConfig, Simulator
    return Simulator(SimConfig(width=40, height=24, radius=1, frames=1, contrast=0.1,
                               mode=lib.ESIM_AD_EXHAUSTIVE, event_capacity=capacity))


@pytest.mark.gpu
def test_events_frame_lookahead_matches_per_frame_drains(lib):
    """Draining frame t after frame t + 1 was pushed (esim_ad_events_frame)
    gives each frame's events exactly as draining after every push."""
    import torch
    from paper_2303_02608_gb300 import EVENT_DTYPE
    frames = _ring_frames(12)
    sim = _ring_sim(lib, 1 << 20)
    ref = []
    for f in frames:
        sim.push(f)
        ref.append(sim.events())
    sim.close()
    sim = _ring_sim(lib, 1 << 20)
    buf = torch.empty(1 << 22, dtype=torch.uint8, pin_memory=True)
    got = []
    sim.push(frames[0])
    for t in range(1, len(frames)):
        sim.push(frames[t])
        n = sim.events_frame_into(t - 1, buf)
        got.append(buf.numpy()[: n * 12].view(EVENT_DTYPE).copy())
    n = sim.events_frame_into(len(frames) - 1, buf)
    got.append(buf.numpy()[: n * 12].view(EVENT_DTYPE).copy())
    sim.close()
    assert sum(len(e) for e in ref) > 1000
    for t, (a, b) in enumerate(zip(ref, got)):
        assert np.array_equal(a, b), t
        assert len(a) == 0 or np.all(a["frame"] == t)


@pytest.mark.gpu
def test_event_ring_wraps(lib):
    """A capacity a little above one frame's events: positions wrap round the
    ring many times over the sequence, and per-frame drains (full or bounded)
    still return every event, in order; three frames left undrained overflow
    it (sticky), the count still covering every event produced."""
    import torch
    from paper_2303_02608_gb300 import EVENT_DTYPE
    frames = _ring_frames(12)
    big = _ring_sim(lib, 1 << 20)
    ref = []
    for f in frames:
        big.push(f)
        ref.append(big.events())
    big.close()
    per_frame = max(len(e) for e in ref)
    cap = per_frame + 37
    for mode in ("full", "frame"):
        sim = _ring_sim(lib, cap)
        buf = torch.empty(cap * 12, dtype=torch.uint8, pin_memory=True)
        for t, f in enumerate(frames):
            sim.push(f)
            if mode == "full":
                got = sim.events()
            else:
                n = sim.events_frame_into(t, buf)
                got = buf.numpy()[: n * 12].view(EVENT_DTYPE).copy()
            assert np.array_equal(got, ref[t]), (mode, t)
        sim.close()
    assert sum(len(e) for e in ref) > 3 * cap      # the ring wrapped
    sim = _ring_sim(lib, cap)
    for f in frames[:4]:
        sim.push(f)                                # frames 1-3 undrained: more than cap
    assert len(ref[1]) + len(ref[2]) + len(ref[3]) > cap
    st, n = lib.esim_ad_events(sim.ctx, 0, 0)
    assert st == lib.ESIM_AD_EOVERFLOW and n == len(ref[1]) + len(ref[2]) + len(ref[3])
    sim.close()


@pytest.mark.gpu
def test_events_frame_arguments(lib):
    import torch
    frames = _ring_frames(10)
    sim = _ring_sim(lib, 1 << 20)
    buf = torch.empty(1 << 20, dtype=torch.uint8, pin_memory=True)
    with pytest.raises(lib.EsimError) as e:
        sim.events_frame_into(0, buf)               # nothing pushed yet
    assert e.value.status == lib.ESIM_AD_EINVAL
    sim.push(frames[0])
    assert sim.events_frame_into(0, buf) == 0       # frame 0 emits nothing
    for f in frames[1:]:
        sim.push(f)
    with pytest.raises(lib.EsimError) as e:
        sim.events_frame_into(1, buf)               # 8 frames behind the latest
    assert e.value.status == lib.ESIM_AD_EINVAL
    n = sim.events_frame_into(5, buf)               # frames 1-5
    assert n > 0 and sim.events_frame_into(3, buf) == 0   # already drained
    rest = sim.events()                             # frames 6-9
    assert len(rest) > 0 and np.all(rest["frame"] >= 6)
    sim.close()
