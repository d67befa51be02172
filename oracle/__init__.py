"""FP64 CPU oracle of the adaptive-denoising event simulator.

TEST INFRASTRUCTURE ONLY: the independent reference the CUDA path is checked
against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
use it; the library never does.  The arithmetic lives in ``esim_oracle.c``
(plain C, double precision, OpenMP over pixels); this module compiles it with
gcc and marshals numpy arrays through ctypes.  ESIM_ORACLE_LIB, when set,
names another build of esim_oracle.c to load instead (the mutation tests load
deliberately broken copies this way, to show that the pins catch them).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esim_oracle.c")
_HDR = os.path.join(_HERE, "esim_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

ADAPTIVE = 0
EXHAUSTIVE = 1


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -O2, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("frames", ctypes.c_int32),
                ("channels", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("pixel_units", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("contrast", ctypes.c_double), ("h", ctypes.c_double),
                ("bandwidth", ctypes.c_double * 7), ("log_eps", ctypes.c_double),
                ("ridge", ctypes.c_double), ("guard_kappa", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(os.environ.get("ESIM_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        lib.or_create.restype = P
        lib.or_create.argtypes = [ctypes.POINTER(_Cfg)]
        lib.or_destroy.argtypes = [P]
        lib.or_push.restype = ctypes.c_int
        lib.or_push.argtypes = [P, P, P, P, P, ctypes.c_int32, ctypes.c_int32]
        lib.or_push_var.restype = ctypes.c_int
        lib.or_push_var.argtypes = [P, P, P, P, P, P, ctypes.c_int32, ctypes.c_int32]
        lib.or_frame_outputs.argtypes = [P, P, P, P, P, P]
        lib.or_event_count.restype = ctypes.c_int64
        lib.or_event_count.argtypes = [P]
        lib.or_take_events.restype = ctypes.c_int64
        lib.or_take_events.argtypes = [P, P, ctypes.c_int64]
        lib.or_get_state.argtypes = [P, P, P, P]
        lib.or_set_state_pixel.argtypes = [P, ctypes.c_int64, ctypes.c_double, P, P]
        lib.or_set_state.argtypes = [P, P, P, P]
        lib.or_wlr_at.restype = ctypes.c_int
        lib.or_wlr_at.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P, P]
        lib.or_threads.restype = ctypes.c_int32
        lib.or_set_threads.argtypes = [ctypes.c_int32]
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().or_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's later calls (timing only)."""
    _load().or_set_threads(int(n))


@dataclass
class OracleConfig:
    width: int
    height: int
    radius: int = 3
    frames: int = 3
    channels: int = 1          # 1 luminance, 3 RGB, 0 radiance already log
    mode: int = ADAPTIVE
    pixel_units: bool = False
    contrast: float = 0.2
    h: float = 1.0
    bandwidth: list = field(default_factory=lambda: [1.0] * 7)
    log_eps: float = 1e-3
    ridge: float = 1e-4
    guard_kappa: float = 0.0   # optional variance guard (extension); <= 0: off


def _f32(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One simulated sequence; push frames in order, read per-frame results."""

    def __init__(self, cfg: OracleConfig):
        self.cfg = cfg
        c = _Cfg()
        c.width, c.height, c.radius, c.frames = cfg.width, cfg.height, cfg.radius, cfg.frames
        c.channels, c.mode, c.pixel_units = cfg.channels, cfg.mode, int(cfg.pixel_units)
        c.contrast, c.h, c.log_eps, c.ridge = cfg.contrast, cfg.h, cfg.log_eps, cfg.ridge
        c.guard_kappa = cfg.guard_kappa
        for j in range(7):
            c.bandwidth[j] = float(cfg.bandwidth[j])
        self._lib = _load()
        self._h = self._lib.or_create(ctypes.byref(c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.n = cfg.width * cfg.height
        self.t = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    def push(self, frame: dict, rows: tuple | None = None) -> None:
        rad = _f32(frame["radiance"])
        nor, alb, dep = _f32(frame["normal"]), _f32(frame["albedo"]), _f32(frame["depth"])
        r0, r1 = (0, -1) if rows is None else rows
        var = frame.get("variance") if self.cfg.guard_kappa > 0 else None
        var = None if var is None else _f32(var)
        rc = self._lib.or_push_var(self._h, _ptr(rad), None if var is None else _ptr(var), _ptr(nor), _ptr(alb),
                                   _ptr(dep), r0, r1)
        if rc != 0:
            raise RuntimeError(f"oracle push failed ({rc})")
        self.t += 1

    def outputs(self) -> dict:
        n = self.n
        H, W = self.cfg.height, self.cfg.width
        alpha, stat, dl = np.empty(n), np.empty(n), np.empty(n)
        nev = np.empty(n, np.int32)
        flag = np.empty(n, np.uint8)
        self._lib.or_frame_outputs(self._h, _ptr(alpha), _ptr(stat), _ptr(dl), _ptr(nev), _ptr(flag))
        return {"alpha": alpha.reshape(H, W), "stat": stat.reshape(H, W), "dl": dl.reshape(H, W),
                "nev": nev.reshape(H, W), "flag": flag.reshape(H, W)}

    def take_events(self) -> np.ndarray:
        k = int(self._lib.or_event_count(self._h))
        out = np.empty((k, 4), np.int32)
        if k:
            self._lib.or_take_events(self._h, _ptr(out), k)
        return out

    def state(self) -> dict:
        n = self.n
        l_last, beta, xc = np.empty(n), np.empty((n, 9)), np.empty((n, 7))
        self._lib.or_get_state(self._h, _ptr(l_last), _ptr(beta), _ptr(xc))
        return {"l_last": l_last, "beta": beta, "xc": xc}

    def set_state_pixel(self, idx: int, l_last: float, beta9, xc7) -> None:
        b = np.ascontiguousarray(beta9, np.float64)
        x = np.ascontiguousarray(xc7, np.float64)
        self._lib.or_set_state_pixel(self._h, int(idx), float(l_last), _ptr(b), _ptr(x))

    def set_state(self, l_last, beta9, xc7) -> None:
        """Overwrite every pixel's model: l_last [n], beta9 [n][9], xc7 [n][7]."""
        n = self.n
        lb = np.ascontiguousarray(np.reshape(l_last, n), np.float64)
        b = np.ascontiguousarray(np.reshape(beta9, (n, 9)), np.float64)
        x = np.ascontiguousarray(np.reshape(xc7, (n, 7)), np.float64)
        self._lib.or_set_state(self._h, _ptr(lb), _ptr(b), _ptr(x))

    def wlr_at(self, cx: int, cy: int):
        theta = np.empty(10)
        R = ctypes.c_double()
        Wd = ctypes.c_double()
        rc = self._lib.or_wlr_at(self._h, cx, cy, _ptr(theta), ctypes.byref(R), ctypes.byref(Wd))
        if rc != 0:
            raise RuntimeError("oracle wlr failed")
        return theta, R.value, Wd.value
