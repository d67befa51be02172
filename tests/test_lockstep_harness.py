"""The lock-step harness that every GPU parity test runs through, checked on
the CPU.  A stand-in for the CUDA simulator is built from a second FP64
oracle (same configuration, float32 outputs like the library's).  Driven
through the harness against the checking oracle it must pass in both
protocols; with a planted discrepancy (alpha off by twice the bar, one event
dropped, polarities flipped, events out of canonical order, one flag
decision reversed) the harness must raise."""
import numpy as np
import pytest
import torch

import lockstep
from oracle import ADAPTIVE, EXHAUSTIVE, Oracle, OracleConfig
from scenes import Scene, preset


class _OracleAsGpu:
    """The surface of paper_2303_02608_gb300.Simulator that the harness uses,
    answered by an FP64 oracle; `fault` plants one discrepancy."""

    def __init__(self, cfg, fault=None):
        self.o = Oracle(cfg)
        self.fault = fault
        self.t = 0

    def push(self, gpu_in):
        self.o.push({k: v.numpy() for k, v in gpu_in.items()})
        self.t += 1

    def denoised(self):
        out = self.o.outputs()
        a = out["alpha"].astype(np.float32)
        f = out["flag"].astype(np.uint8)
        if self.fault == "alpha" and self.t > 1:
            a = a + np.float32(2 * lockstep.ALPHA_TOL)
        if self.fault == "flag" and self.t > 1:
            idx = np.unravel_index(np.argmin(f), f.shape) if (f == 0).any() else (0, 0)
            f[idx] ^= 1
        return torch.from_numpy(a), torch.from_numpy(f)

    def events(self):
        from paper_2303_02608_gb300 import EVENT_DTYPE
        ev = self.o.take_events()
        out = np.zeros(len(ev), EVENT_DTYPE)
        if len(ev):
            out["frame"], out["x"], out["y"], out["polarity"] = ev[:, 0], ev[:, 1], ev[:, 2], ev[:, 3]
        if len(out) > 1:
            if self.fault == "drop":
                out = out[:-1]
            elif self.fault == "polarity":
                out["polarity"] = -out["polarity"]
            elif self.fault == "order":
                out = out[::-1].copy()
        return out

    def get_state(self):
        st = self.o.state()
        return {"l_last": st["l_last"].astype(np.float32), "beta": st["beta"][:, 2:].astype(np.float32),
                "xc": st["xc"].astype(np.float32)}


@pytest.fixture
def cpu_tensors(monkeypatch):
    # the harness moves inputs to the device and synchronises; here both are no-ops
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def _case(mode, fault=None, strict=True):
    cfg_s = preset("disc64", frames=6)
    frames = Scene(cfg_s).sequence()
    ocfg = OracleConfig(cfg_s.width, cfg_s.height, radius=3, frames=3, channels=1, mode=mode, contrast=0.2)
    gpu = _OracleAsGpu(ocfg, fault)
    return lockstep.run(frames, gpu, Oracle(ocfg), 0.2, strict=strict, adaptive=(mode == ADAPTIVE))


@pytest.mark.parametrize("mode", [ADAPTIVE, EXHAUSTIVE])
@pytest.mark.parametrize("strict", [True, False])
def test_honest_stand_in_passes(cpu_tensors, mode, strict):
    rep = _case(mode, strict=strict)
    assert rep["frames"] == 6 and rep["events"] > 0 and rep["regressed"] > 0
    assert rep["alpha_max_err"] < 1e-6        # float32 rounding of alpha only
    # decisions excused only where float32 rounding of the model can move them
    assert rep["flag_ambiguous"] + rep["event_ambiguous"] <= 0.001 * rep["regressed"] + 2


@pytest.mark.parametrize("fault", ["alpha", "drop", "polarity", "order", "flag"])
def test_planted_discrepancy_fails(cpu_tensors, fault):
    with pytest.raises(AssertionError):
        _case(ADAPTIVE, fault)
