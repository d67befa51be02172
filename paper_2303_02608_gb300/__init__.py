"""Python binding of libesim_ad (the C ABI in include/esim_ad.h).

Argument marshalling only: every step of the simulator runs in the CUDA
library.  The functions keep the C names; ``Simulator`` wraps a context with
torch tensors for device memory and streams.  Importing this module does not
touch the GPU; the first call loads ``libesim_ad.so`` from this directory and
raises if it has not been built (``python -m paper_2303_02608_gb300.build``).
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libesim_ad.so")

ESIM_AD_OK = 0
ESIM_AD_EINVAL = -1
ESIM_AD_ENOMEM = -2
ESIM_AD_ECUDA = -3
ESIM_AD_EOVERFLOW = -4
ESIM_AD_ETIMEOUT = -5
ESIM_AD_ESTATE = -6
ESIM_AD_ENOSPACE = -7

ESIM_AD_ADAPTIVE = 0
ESIM_AD_EXHAUSTIVE = 1
ESIM_AD_LUMA_F32 = 0
ESIM_AD_RGB_F32 = 1
ESIM_AD_LOGLUMA_F16 = 2
ESIM_AD_FEAT_F32 = 0
ESIM_AD_FEAT_BF16 = 1
ESIM_AD_FP32 = 0
ESIM_AD_MIXED = 1

# Every exported symbol of the library, as declared in include/esim_ad.h.
EXPORTS = (
    "esim_ad_init", "esim_ad_push_frame", "esim_ad_events", "esim_ad_events_frame", "esim_ad_denoised",
    "esim_ad_get_state", "esim_ad_set_state", "esim_ad_reset", "esim_ad_stats_get",
    "esim_ad_destroy", "esim_ad_status_string", "esim_ad_profile_enable", "esim_ad_profile_get",
    "esim_ad_write_events_noalloc", "esim_ad_batch_tiling", "esim_ad_wlr_workspace_size", "esim_ad_wlr_forward",
    "esim_ad_wlr_backward", "esim_ad_batch_init", "esim_ad_batch_step", "esim_ad_batch_events",
    "esim_ad_batch_reset_sequence", "esim_ad_batch_denoised", "esim_ad_batch_get_state",
    "esim_ad_batch_stats", "esim_ad_batch_profile_enable", "esim_ad_batch_profile_get",
    "esim_ad_batch_destroy", "esim_ad_esim_frame", "esim_ad_quality_workspace_size", "esim_ad_quality",
    "esim_ad_render", "esim_ad_wlr2_workspace_size", "esim_ad_wlr2_forward",
)


class esim_ad_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("radius", ctypes.c_int32), ("frames", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("radiance_fmt", ctypes.c_int32), ("feature_fmt", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("contrast", ctypes.c_float), ("h", ctypes.c_float), ("bandwidth", ctypes.c_float * 7),
        ("log_eps", ctypes.c_float), ("ridge", ctypes.c_float), ("feature_scale", ctypes.c_float * 7),
        ("guard_kappa", ctypes.c_float), ("event_capacity", ctypes.c_uint64),
    ]


class esim_ad_frame(ctypes.Structure):
    _fields_ = [
        ("radiance", ctypes.c_void_p), ("variance", ctypes.c_void_p), ("normal", ctypes.c_void_p),
        ("albedo", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("features", ctypes.c_void_p),
        ("on_host", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("pitch_elems", ctypes.c_int64),
    ]


class esim_ad_stats(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_uint64), ("regressions", ctypes.c_uint64),
                ("events", ctypes.c_uint64), ("pixels", ctypes.c_uint64), ("fp64_solves", ctypes.c_uint64),
                ("staged_ingests", ctypes.c_uint64)]


class esim_ad_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 3), ("kernels", ctypes.c_uint64), ("ms", ctypes.c_double * 3),
                ("neighbours", ctypes.c_uint64), ("regressions", ctypes.c_uint64)]


class esim_ad_wlr_desc(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("sequence", ctypes.c_int32), ("radius", ctypes.c_int32), ("frames", ctypes.c_int32),
                ("radiance_fmt", ctypes.c_int32), ("h", ctypes.c_float), ("log_eps", ctypes.c_float),
                ("ridge", ctypes.c_float)]


BATCH_EVENT_DTYPE = np.dtype({"names": ["frame", "x", "y", "polarity", "seq"],
                              "formats": ["<u4", "<u2", "<u2", "i1", "<u2"],
                              "offsets": [0, 4, 6, 8, 10], "itemsize": 12})

EVENT_DTYPE = np.dtype({"names": ["frame", "x", "y", "polarity"],
                        "formats": ["<u4", "<u2", "<u2", "i1"],
                        "offsets": [0, 4, 6, 8], "itemsize": 12})


class EsimError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lib = None


def load_library():
    """Load libesim_ad.so from this package directory (fails loudly if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2303_02608_gb300.build`"
                          " (the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    st = ctypes.c_int
    lib.esim_ad_init.restype = st
    lib.esim_ad_init.argtypes = [ctypes.POINTER(esim_ad_config), P, ctypes.POINTER(P)]
    lib.esim_ad_push_frame.restype = st
    lib.esim_ad_push_frame.argtypes = [P, ctypes.POINTER(esim_ad_frame)]
    lib.esim_ad_events.restype = st
    lib.esim_ad_events.argtypes = [P, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
    lib.esim_ad_events_frame.restype = st
    lib.esim_ad_events_frame.argtypes = [P, ctypes.c_uint64, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.c_int]
    lib.esim_ad_denoised.restype = st
    lib.esim_ad_denoised.argtypes = [P, P, P, ctypes.c_int]
    lib.esim_ad_get_state.restype = st
    lib.esim_ad_get_state.argtypes = [P, P, P, P]
    lib.esim_ad_set_state.restype = st
    lib.esim_ad_set_state.argtypes = [P, P, P, P]
    lib.esim_ad_reset.restype = st
    lib.esim_ad_reset.argtypes = [P]
    lib.esim_ad_stats_get.restype = st
    lib.esim_ad_stats_get.argtypes = [P, ctypes.POINTER(esim_ad_stats)]
    lib.esim_ad_destroy.restype = None
    lib.esim_ad_destroy.argtypes = [P]
    lib.esim_ad_profile_enable.restype = st
    lib.esim_ad_profile_enable.argtypes = [P, ctypes.c_int]
    lib.esim_ad_profile_get.restype = st
    lib.esim_ad_profile_get.argtypes = [P, ctypes.POINTER(esim_ad_profile)]
    lib.esim_ad_batch_tiling.restype = st
    lib.esim_ad_batch_tiling.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32)]
    lib.esim_ad_write_events_noalloc.restype = st
    lib.esim_ad_write_events_noalloc.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, P,
                                                 ctypes.c_uint64, P, P]
    lib.esim_ad_wlr_workspace_size.restype = ctypes.c_size_t
    lib.esim_ad_wlr_workspace_size.argtypes = [ctypes.POINTER(esim_ad_wlr_desc)]
    lib.esim_ad_wlr_forward.restype = st
    lib.esim_ad_wlr_forward.argtypes = [ctypes.POINTER(esim_ad_wlr_desc), P, P, P, P, P, P, P]
    lib.esim_ad_wlr2_workspace_size.restype = ctypes.c_size_t
    lib.esim_ad_wlr2_workspace_size.argtypes = [ctypes.POINTER(esim_ad_wlr_desc)]
    lib.esim_ad_wlr2_forward.restype = st
    lib.esim_ad_wlr2_forward.argtypes = [ctypes.POINTER(esim_ad_wlr_desc), P, P, P, P, P, P]
    lib.esim_ad_wlr_backward.restype = st
    lib.esim_ad_wlr_backward.argtypes = [ctypes.POINTER(esim_ad_wlr_desc), P, P, P, P, P, P, P, P, P]
    lib.esim_ad_batch_init.restype = st
    lib.esim_ad_batch_init.argtypes = [ctypes.POINTER(esim_ad_config), ctypes.c_int32, P, ctypes.POINTER(P)]
    lib.esim_ad_batch_step.restype = st
    lib.esim_ad_batch_step.argtypes = [P, ctypes.POINTER(esim_ad_frame)]
    lib.esim_ad_batch_events.restype = st
    lib.esim_ad_batch_events.argtypes = [P, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
    lib.esim_ad_batch_reset_sequence.restype = st
    lib.esim_ad_batch_reset_sequence.argtypes = [P, ctypes.c_int32]
    lib.esim_ad_batch_denoised.restype = st
    lib.esim_ad_batch_denoised.argtypes = [P, ctypes.c_int32, P, P, ctypes.c_int]
    lib.esim_ad_batch_get_state.restype = st
    lib.esim_ad_batch_get_state.argtypes = [P, ctypes.c_int32, P, P, P]
    lib.esim_ad_batch_stats.restype = st
    lib.esim_ad_batch_stats.argtypes = [P, ctypes.POINTER(esim_ad_stats), ctypes.POINTER(ctypes.c_int32)]
    lib.esim_ad_batch_profile_enable.restype = st
    lib.esim_ad_batch_profile_enable.argtypes = [P, ctypes.c_int]
    lib.esim_ad_batch_profile_get.restype = st
    lib.esim_ad_batch_profile_get.argtypes = [P, ctypes.POINTER(esim_ad_profile)]
    lib.esim_ad_batch_destroy.restype = None
    lib.esim_ad_batch_destroy.argtypes = [P]
    lib.esim_ad_esim_frame.restype = st
    lib.esim_ad_esim_frame.argtypes = [P, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_int32, P, P,
                                       ctypes.c_int64, P]
    lib.esim_ad_quality_workspace_size.restype = ctypes.c_size_t
    lib.esim_ad_quality_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.esim_ad_quality.restype = st
    lib.esim_ad_quality.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P,
                                    ctypes.c_size_t, ctypes.POINTER(esim_ad_quality_result), P]
    lib.esim_ad_render.restype = st
    lib.esim_ad_render.argtypes = [ctypes.POINTER(esim_ad_render_scene), ctypes.c_int32, P, P, P, P, P, P]
    lib.esim_ad_status_string.restype = ctypes.c_char_p
    lib.esim_ad_status_string.argtypes = [st]
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load_library().esim_ad_status_string(int(status)).decode()
    except ImportError:
        return "library not loaded"


def _check(status: int, what: str) -> None:
    if status != ESIM_AD_OK:
        raise EsimError(status, what)


# ------------------------------------------------------------- C-named calls

def make_config(width: int, height: int, radius: int = 7, frames: int = 5, contrast: float = 0.15,
                mode: int = ESIM_AD_ADAPTIVE, rgb: bool = True, h: float = 1.0, bandwidth=None,
                log_eps: float = 1e-3, ridge: float = 1e-4, event_capacity: int = 1 << 22,
                radiance_fmt: int | None = None, feature_fmt: int = ESIM_AD_FEAT_F32,
                precision: int = ESIM_AD_FP32, feature_scale=None, guard_kappa: float = 0.0) -> esim_ad_config:
    c = esim_ad_config()
    c.struct_size = ctypes.sizeof(esim_ad_config)
    c.width, c.height, c.radius, c.frames = width, height, radius, frames
    c.mode = mode
    if radiance_fmt is None:
        radiance_fmt = ESIM_AD_RGB_F32 if rgb else ESIM_AD_LUMA_F32
    c.radiance_fmt, c.feature_fmt, c.precision = radiance_fmt, feature_fmt, precision
    fs = [1.0] * 7 if feature_scale is None else list(feature_scale)
    for j in range(7):
        c.feature_scale[j] = float(fs[j])
    c.contrast, c.h, c.log_eps, c.ridge = contrast, h, log_eps, ridge
    bw = [1.0] * 7 if bandwidth is None else list(bandwidth)
    for j in range(7):
        c.bandwidth[j] = float(bw[j])
    c.event_capacity = int(event_capacity)
    c.guard_kappa = float(guard_kappa)
    return c


def esim_ad_init(cfg: esim_ad_config, cuda_stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load_library().esim_ad_init(ctypes.byref(cfg), ctypes.c_void_p(cuda_stream or None),
                                        ctypes.byref(h)), "esim_ad_init")
    return h.value


def esim_ad_push_frame(ctx: int, radiance: int, normal: int = 0, albedo: int = 0, depth: int = 0,
                       variance: int = 0, on_host: bool = False, features: int = 0, pitch: int = 0) -> None:
    f = esim_ad_frame(radiance, variance or None, normal or None, albedo or None, depth or None,
                      features or None, int(on_host), 0, int(pitch))
    _check(load_library().esim_ad_push_frame(ctypes.c_void_p(ctx), ctypes.byref(f)), "esim_ad_push_frame")


def esim_ad_events(ctx: int, dst: int, cap: int, dst_is_device: bool = False) -> tuple[int, int]:
    """Returns (status, n).  Status is returned, not raised, because ENOSPACE
    and EOVERFLOW carry a count."""
    n = ctypes.c_uint64(0)
    st = load_library().esim_ad_events(ctypes.c_void_p(ctx), ctypes.c_void_p(dst or None),
                                       ctypes.c_uint64(cap), ctypes.byref(n), int(dst_is_device))
    return st, n.value


def esim_ad_events_frame(ctx: int, frame: int, dst: int, cap: int, dst_is_device: bool = False) -> tuple[int, int]:
    """Drain the events of frames up to `frame`; returns (status, n) like esim_ad_events."""
    n = ctypes.c_uint64(0)
    st = load_library().esim_ad_events_frame(ctypes.c_void_p(ctx), ctypes.c_uint64(frame), ctypes.c_void_p(dst or None),
                                             ctypes.c_uint64(cap), ctypes.byref(n), int(dst_is_device))
    return st, n.value


def esim_ad_denoised(ctx: int, alpha: int, flags: int, dst_is_device: bool = True) -> None:
    _check(load_library().esim_ad_denoised(ctypes.c_void_p(ctx), ctypes.c_void_p(alpha or None),
                                           ctypes.c_void_p(flags or None), int(dst_is_device)),
           "esim_ad_denoised")


def esim_ad_get_state(ctx: int, l_last: int, beta: int, xc: int) -> None:
    _check(load_library().esim_ad_get_state(ctypes.c_void_p(ctx), ctypes.c_void_p(l_last or None),
                                            ctypes.c_void_p(beta or None), ctypes.c_void_p(xc or None)),
           "esim_ad_get_state")


def esim_ad_set_state(ctx: int, l_last: int, beta: int, xc: int) -> None:
    _check(load_library().esim_ad_set_state(ctypes.c_void_p(ctx), ctypes.c_void_p(l_last or None),
                                            ctypes.c_void_p(beta or None), ctypes.c_void_p(xc or None)),
           "esim_ad_set_state")


def esim_ad_reset(ctx: int) -> None:
    _check(load_library().esim_ad_reset(ctypes.c_void_p(ctx)), "esim_ad_reset")


def esim_ad_stats_get(ctx: int) -> dict:
    s = esim_ad_stats()
    _check(load_library().esim_ad_stats_get(ctypes.c_void_p(ctx), ctypes.byref(s)), "esim_ad_stats_get")
    return {"frames": s.frames, "regressions": s.regressions, "events": s.events, "pixels": s.pixels,
            "fp64_solves": s.fp64_solves, "staged_ingests": s.staged_ingests}


def esim_ad_profile_enable(ctx: int, on: bool = True) -> None:
    _check(load_library().esim_ad_profile_enable(ctypes.c_void_p(ctx), int(on)), "esim_ad_profile_enable")


KERNEL_CLASSES = ("ingest_test", "wlr_emit", "event_write")


def esim_ad_profile_get(ctx: int) -> dict:
    p = esim_ad_profile()
    _check(load_library().esim_ad_profile_get(ctypes.c_void_p(ctx), ctypes.byref(p)), "esim_ad_profile_get")
    return {"launches": {k: int(p.launches[i]) for i, k in enumerate(KERNEL_CLASSES)},
            "ms": {k: float(p.ms[i]) for i, k in enumerate(KERNEL_CLASSES)},
            "kernels": int(p.kernels), "neighbours": int(p.neighbours), "regressions": int(p.regressions)}


def esim_ad_write_events_noalloc(counts: int, width: int, height: int, frame: int, events: int,
                                 capacity: int, total_device: int, cuda_stream: int = 0) -> int:
    """Allocation-free event writer (device pointers in and out); returns the status."""
    return load_library().esim_ad_write_events_noalloc(
        ctypes.c_void_p(counts or None), width, height, frame, ctypes.c_void_p(events or None),
        ctypes.c_uint64(capacity), ctypes.c_void_p(total_device or None), ctypes.c_void_p(cuda_stream or None))


class esim_ad_sphere(ctypes.Structure):
    _fields_ = [("center", ctypes.c_float * 3), ("velocity", ctypes.c_float * 3), ("radius", ctypes.c_float),
                ("albedo", ctypes.c_float * 3)]


class esim_ad_render_scene(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("spp", ctypes.c_int32), ("max_bounces", ctypes.c_int32), ("n_spheres", ctypes.c_int32),
                ("seed", ctypes.c_uint32), ("cam_pos", ctypes.c_float * 3), ("tan_half_fov_y", ctypes.c_float),
                ("box", ctypes.c_float * 3), ("wall_albedo", (ctypes.c_float * 3) * 5),
                ("back_albedo2", ctypes.c_float * 3), ("checker", ctypes.c_float), ("light", ctypes.c_float * 4),
                ("light_radiance", ctypes.c_float * 3), ("eps", ctypes.c_float),
                ("spheres", esim_ad_sphere * 8)]


def make_render_scene(sc) -> esim_ad_render_scene:
    """C description of a scenes.cornell.RenderScene."""
    r = esim_ad_render_scene()
    r.struct_size = ctypes.sizeof(esim_ad_render_scene)
    r.width, r.height, r.spp, r.max_bounces = sc.width, sc.height, sc.spp, sc.max_bounces
    r.n_spheres, r.seed = len(sc.spheres), sc.seed
    r.cam_pos[:] = list(sc.cam_pos)
    r.tan_half_fov_y = sc.tan_half_fov_y
    r.box[:] = list(sc.box)
    for k in range(5):
        r.wall_albedo[k][:] = list(sc.wall_albedo[k])
    r.back_albedo2[:] = list(sc.back_albedo2)
    r.checker = sc.checker
    r.light[:] = list(sc.light)
    r.light_radiance[:] = list(sc.light_radiance)
    r.eps = sc.eps
    for j, sp in enumerate(sc.spheres):
        r.spheres[j].center[:] = list(sp.center)
        r.spheres[j].velocity[:] = list(sp.velocity)
        r.spheres[j].radius = sp.radius
        r.spheres[j].albedo[:] = list(sp.albedo)
    return r


def render(sc, frame: int, device=None) -> dict:
    """Render one frame of a test scene on the GPU: radiance [3][H][W],
    variance [H][W], normal [3][H][W], albedo [3][H][W], depth [H][W]
    (float32 CUDA tensors, the simulator's input format)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    H, W = sc.height, sc.width
    out = {"radiance": torch.empty(3, H, W, device=dev), "variance": torch.empty(H, W, device=dev),
           "normal": torch.empty(3, H, W, device=dev), "albedo": torch.empty(3, H, W, device=dev),
           "depth": torch.empty(H, W, device=dev)}
    desc = make_render_scene(sc)
    _check(load_library().esim_ad_render(ctypes.byref(desc), int(frame),
                                         *(ctypes.c_void_p(out[k].data_ptr()) for k in
                                           ("radiance", "variance", "normal", "albedo", "depth")),
                                         ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)),
           "esim_ad_render")
    return out


class esim_ad_quality_result(ctypes.Structure):
    _fields_ = [("n_tau", ctypes.c_int32), ("tau", ctypes.c_float * 16), ("precision", ctypes.c_double * 16),
                ("recall", ctypes.c_double * 16), ("fscore", ctypes.c_double * 16), ("chamfer", ctypes.c_double),
                ("n_gen", ctypes.c_uint64), ("n_ref", ctypes.c_uint64)]


def esim_frame(radiance, l_last, counts, contrast: float, init: bool, log_eps: float = 1e-3) -> None:
    """One frame of plain ESIM (the evaluation's reference and baseline
    simulator) on device tensors: radiance [C][H][W] float32 (C = 1 or 3),
    l_last [H][W] float32 (in/out), counts [H][W] int32 (out)."""
    import torch
    for t, dt in ((radiance, torch.float32), (l_last, torch.float32), (counts, torch.int32)):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError("esim_frame: contiguous device tensors of the documented types")
    n = l_last.numel()
    if radiance.numel() != radiance.shape[0] * n or counts.numel() != n:
        raise ValueError("esim_frame: shapes do not match")
    _check(load_library().esim_ad_esim_frame(
        ctypes.c_void_p(radiance.data_ptr()), radiance.shape[0], log_eps, contrast, int(init),
        ctypes.c_void_p(l_last.data_ptr()), ctypes.c_void_p(counts.data_ptr()), n,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "esim_ad_esim_frame")


def quality(gen, ref, taus) -> dict:
    """P(tau), R(tau), F(tau) and the chamfer distance of generated events
    against reference events, both signed count maps [F][H][W] int32 on the
    device (the workspace comes from torch)."""
    import torch
    if gen.shape != ref.shape or gen.dim() != 3:
        raise ValueError("quality: two [F][H][W] count maps of one shape")
    for t in (gen, ref):
        if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
            raise ValueError("quality: contiguous int32 device tensors")
    F, H, W = gen.shape
    lib = load_library()
    ws_bytes = int(lib.esim_ad_quality_workspace_size(W, H, F))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=gen.device)
    tau = (ctypes.c_float * len(taus))(*taus)
    r = esim_ad_quality_result()
    _check(lib.esim_ad_quality(ctypes.c_void_p(gen.data_ptr()), ctypes.c_void_p(ref.data_ptr()), W, H, F, tau,
                               len(taus), ctypes.c_void_p(ws.data_ptr()), ws_bytes, ctypes.byref(r),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "esim_ad_quality")
    k = r.n_tau
    return {"tau": list(r.tau[:k]), "precision": list(r.precision[:k]), "recall": list(r.recall[:k]),
            "fscore": list(r.fscore[:k]), "chamfer": r.chamfer, "n_gen": int(r.n_gen), "n_ref": int(r.n_ref)}


def make_wlr_desc(width: int, height: int, sequence: int, radius: int = 3, frames: int = 3, rgb: bool = True,
                  h: float = 1.0, log_eps: float = 1e-3, ridge: float = 1e-4) -> esim_ad_wlr_desc:
    d = esim_ad_wlr_desc()
    d.struct_size = ctypes.sizeof(esim_ad_wlr_desc)
    d.width, d.height, d.sequence, d.radius, d.frames = width, height, sequence, radius, frames
    d.radiance_fmt = ESIM_AD_RGB_F32 if rgb else ESIM_AD_LUMA_F32
    d.h, d.log_eps, d.ridge = h, log_eps, ridge
    return d


def esim_ad_wlr_workspace_size(desc: esim_ad_wlr_desc) -> int:
    return int(load_library().esim_ad_wlr_workspace_size(ctypes.byref(desc)))


def esim_ad_wlr_forward(desc, radiance: int, features: int, bandwidth: int, alpha: int, saved: int,
                        workspace: int, cuda_stream: int = 0) -> None:
    _check(load_library().esim_ad_wlr_forward(ctypes.byref(desc), *(ctypes.c_void_p(x) for x in (
        radiance, features, bandwidth, alpha, saved, workspace, cuda_stream or None))), "esim_ad_wlr_forward")


def esim_ad_wlr_backward(desc, radiance: int, features: int, bandwidth: int, saved: int, g_alpha: int,
                         g_radiance: int, g_bandwidth: int, workspace: int, cuda_stream: int = 0) -> None:
    _check(load_library().esim_ad_wlr_backward(ctypes.byref(desc), *(ctypes.c_void_p(x) for x in (
        radiance, features, bandwidth, saved, g_alpha, g_radiance, g_bandwidth, workspace,
        cuda_stream or None))), "esim_ad_wlr_backward")


def esim_ad_wlr2_workspace_size(desc: esim_ad_wlr_desc) -> int:
    return int(load_library().esim_ad_wlr2_workspace_size(ctypes.byref(desc)))


def esim_ad_wlr2_forward(desc, radiance: int, features: int, bandwidth: int, alpha: int, workspace: int,
                         cuda_stream: int = 0) -> None:
    _check(load_library().esim_ad_wlr2_forward(ctypes.byref(desc), *(ctypes.c_void_p(x) for x in (
        radiance, features, bandwidth, alpha, workspace, cuda_stream or None))), "esim_ad_wlr2_forward")


def wlr2(radiance, features, bandwidth=None, radius: int = 3, frames: int = 3, h: float = 1.0,
         log_eps: float = 1e-3, ridge: float = 1e-4, workspace=None):
    """Second-order dense regression: radiance [F][C][H][W], features [F][7][H][W]
    (normal xyz, depth, albedo rgb), bandwidth [7] (default all 1) -> alpha
    [F][H][W], all float32 device tensors.  `workspace` (uint8, at least
    esim_ad_wlr2_workspace_size bytes) may be passed to reuse one across calls."""
    import torch
    F_, C, H, W = radiance.shape
    if C not in (1, 3) or features.shape != (F_, 7, H, W):
        raise ValueError("wlr2: radiance [F][1|3][H][W] and features [F][7][H][W]")
    dev = radiance.device
    if bandwidth is None:
        bandwidth = torch.ones(7, dtype=torch.float32, device=dev)
    radiance, features, bandwidth = (t.contiguous().float() for t in (radiance, features, bandwidth))
    desc = make_wlr_desc(W, H, F_, radius, frames, C == 3, h, log_eps, ridge)
    need = esim_ad_wlr2_workspace_size(desc)
    if need == 0:
        raise ValueError("wlr2: invalid sizes or parameters")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    alpha = torch.empty(F_, H, W, dtype=torch.float32, device=dev)
    esim_ad_wlr2_forward(desc, radiance.data_ptr(), features.data_ptr(), bandwidth.data_ptr(), alpha.data_ptr(),
                         workspace.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    return alpha


def _wlr_function():
    import torch

    class WLRFunction(torch.autograd.Function):
        """alpha = WLR(radiance, features; bandwidth): the dense regression of every
        pixel of every frame, differentiable in the radiance and the 7 feature
        bandwidths.  Forward and backward run in the library's kernels."""

        @staticmethod
        def forward(ctx, radiance, features, bandwidth, radius, frames, h, log_eps, ridge):
            F_, C, H, W = radiance.shape
            desc = make_wlr_desc(W, H, F_, radius, frames, C == 3, h, log_eps, ridge)
            dev = radiance.device
            ws = torch.empty(esim_ad_wlr_workspace_size(desc), dtype=torch.uint8, device=dev)
            alpha = torch.empty(F_, H, W, dtype=torch.float32, device=dev)
            saved = torch.empty(F_, 20, H, W, dtype=torch.float32, device=dev)
            radiance, features, bandwidth = (t.contiguous().float() for t in (radiance, features, bandwidth))
            stream = torch.cuda.current_stream(dev).cuda_stream
            esim_ad_wlr_forward(desc, radiance.data_ptr(), features.data_ptr(), bandwidth.data_ptr(),
                                alpha.data_ptr(), saved.data_ptr(), ws.data_ptr(), stream)
            ctx.desc = desc
            ctx.save_for_backward(radiance, features, bandwidth, saved, ws)
            return alpha

        @staticmethod
        def backward(ctx, g_alpha):
            radiance, features, bandwidth, saved, ws = ctx.saved_tensors
            g_alpha = g_alpha.contiguous().float()
            g_rad = torch.empty_like(radiance)
            g_b = torch.empty(7, dtype=torch.float32, device=radiance.device)
            stream = torch.cuda.current_stream(radiance.device).cuda_stream
            esim_ad_wlr_backward(ctx.desc, radiance.data_ptr(), features.data_ptr(), bandwidth.data_ptr(),
                                 saved.data_ptr(), g_alpha.data_ptr(), g_rad.data_ptr(), g_b.data_ptr(),
                                 ws.data_ptr(), stream)
            return g_rad, None, g_b, None, None, None, None, None

    return WLRFunction


_WLR = None


def wlr(radiance, features, bandwidth, radius: int = 3, frames: int = 3, h: float = 1.0, log_eps: float = 1e-3,
        ridge: float = 1e-4):
    """Differentiable dense regression: radiance [F][C][H][W], features [F][7][H][W]
    (normal xyz, depth, albedo rgb), bandwidth [7] -> alpha [F][H][W]."""
    global _WLR
    if _WLR is None:
        _WLR = _wlr_function()
    return _WLR.apply(radiance, features, bandwidth, radius, frames, h, log_eps, ridge)


def esim_ad_destroy(ctx: int) -> None:
    if ctx:
        load_library().esim_ad_destroy(ctypes.c_void_p(ctx))


# ------------------------------------------------------------- convenience

@dataclass
class SimConfig:
    width: int
    height: int
    radius: int = 7
    frames: int = 5
    contrast: float = 0.15
    mode: int = ESIM_AD_ADAPTIVE
    rgb: bool = True
    h: float = 1.0
    bandwidth: list = field(default_factory=lambda: [1.0] * 7)
    log_eps: float = 1e-3
    ridge: float = 1e-4
    event_capacity: int = 1 << 22
    radiance_fmt: int | None = None      # default: RGB_F32 if rgb else LUMA_F32
    feature_fmt: int = ESIM_AD_FEAT_F32
    precision: int = ESIM_AD_FP32
    feature_scale: list = field(default_factory=lambda: [1.0] * 7)
    guard_kappa: float = 0.0             # optional variance guard of the test; <= 0: off

    def c_config(self) -> esim_ad_config:
        return make_config(self.width, self.height, self.radius, self.frames, self.contrast, self.mode,
                           self.rgb, self.h, self.bandwidth, self.log_eps, self.ridge, self.event_capacity,
                           self.radiance_fmt, self.feature_fmt, self.precision, self.feature_scale,
                           self.guard_kappa)


class Simulator:
    """One event-simulation context on the current CUDA device and stream.

    ``push`` accepts a dict with ``radiance`` ([C][H][W] float32, or [H][W]
    float16 log brightness) and either ``normal`` [3][H][W], ``albedo``
    [3][H][W], ``depth`` [H][W] float32 or ``features`` [7][H][W] bfloat16, as
    contiguous torch tensors, all on the GPU or all on the host (pinned for
    asynchronous copies).
    """

    def __init__(self, cfg: SimConfig, stream=None):
        import torch
        self.cfg = cfg
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = esim_ad_init(cfg.c_config(), self.stream.cuda_stream)
        self._keep = []
        self._t = 0            # index of the next frame pushed
        self._ev_host = None   # pinned landing buffer of events(), grown on demand

    def close(self):
        if getattr(self, "ctx", None):
            esim_ad_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def push(self, frame: dict, pitch: int = 0) -> None:
        """Push one frame: planes [C][H][W] (or [C][H][pitch] with only the first
        W columns read, when pitch is given)."""
        t = self._torch
        keys = ["radiance"] + (["features"] if "features" in frame else ["normal", "albedo", "depth"])
        if self.cfg.guard_kappa > 0 and frame.get("variance") is not None:
            keys.append("variance")
        planes = [frame[k] for k in keys]
        on_host = not planes[0].is_cuda
        for p in planes:
            if p.dtype not in (t.float32, t.float16, t.bfloat16) or not p.is_contiguous() or p.is_cuda == on_host:
                raise ValueError("frame planes must be contiguous, all on the GPU or all on the host")
        ptr = {k: v.data_ptr() for k, v in zip(keys, planes)}
        esim_ad_push_frame(self.ctx, ptr["radiance"], ptr.get("normal", 0), ptr.get("albedo", 0),
                           ptr.get("depth", 0), variance=ptr.get("variance", 0), on_host=on_host,
                           features=ptr.get("features", 0), pitch=pitch)
        # inputs (device planes, or pinned host planes copied asynchronously) are
        # read in stream order; keep them alive until a sync point covers them
        self._keep.append((self._t, planes))
        self._t += 1

    def events(self) -> np.ndarray:
        """Drain the events produced so far (one synchronising call when they
        fit the pinned landing buffer, which grows to the largest drain)."""
        t = self._torch
        buf = self._ev_host
        cap = 0 if buf is None else buf.numel() // EVENT_DTYPE.itemsize
        st, n = esim_ad_events(self.ctx, buf.data_ptr() if cap else 0, cap)
        if st == ESIM_AD_ENOSPACE:
            cap = max(n, 2 * cap, 1 << 16)
            self._ev_host = buf = t.empty(cap * EVENT_DTYPE.itemsize, dtype=t.uint8, pin_memory=True)
            st, n = esim_ad_events(self.ctx, buf.data_ptr(), cap)
        _check(st, "esim_ad_events")
        out = np.empty(n, EVENT_DTYPE)
        if n:
            out.view(np.uint8)[:] = buf.numpy()[: n * EVENT_DTYPE.itemsize]
        self._keep.clear()
        return out

    def events_into(self, dst) -> int:
        """Drain the events produced so far into `dst`, a tensor owned by the
        caller (pinned host memory, or device memory), as 12-byte records of
        EVENT_DTYPE; returns their number.  One synchronising call and one
        copy, no array allocated; raises EsimError (ENOSPACE) when they do not
        fit, draining nothing."""
        cap = dst.numel() * dst.element_size() // EVENT_DTYPE.itemsize
        st, n = esim_ad_events(self.ctx, dst.data_ptr(), cap, dst_is_device=bool(dst.is_cuda))
        _check(st, "esim_ad_events")
        self._keep.clear()
        return n

    def events_frame_into(self, frame: int, dst) -> int:
        """Drain the events of the frames up to `frame` (the index of a pushed
        frame, at most 7 behind the latest) into the caller's tensor `dst`
        (pinned host or device memory); waits for that frame's event writer
        only, so the frames pushed after it keep running.  Returns the number
        of events; raises EsimError (ENOSPACE) when they do not fit."""
        cap = dst.numel() * dst.element_size() // EVENT_DTYPE.itemsize
        st, n = esim_ad_events_frame(self.ctx, frame, dst.data_ptr(), cap, dst_is_device=bool(dst.is_cuda))
        _check(st, "esim_ad_events_frame")
        self._keep = [e for e in self._keep if e[0] > frame]   # frames up to `frame` are done
        return n

    def events_device(self, dst, cap: int) -> int:
        st, n = esim_ad_events(self.ctx, dst.data_ptr(), cap, dst_is_device=True)
        _check(st, "esim_ad_events")
        self._keep.clear()
        return n

    def denoised(self):
        t = self._torch
        a = t.empty(self.cfg.height, self.cfg.width, dtype=t.float32, device=self.device)
        f = t.empty(self.cfg.height, self.cfg.width, dtype=t.uint8, device=self.device)
        esim_ad_denoised(self.ctx, a.data_ptr(), f.data_ptr(), True)
        return a, f

    def get_state(self) -> dict:
        n = self.cfg.width * self.cfg.height
        l_last = np.empty(n, np.float32)
        beta = np.empty((n, 7), np.float32)
        xc = np.empty((n, 7), np.float32)
        esim_ad_get_state(self.ctx, l_last.ctypes.data, beta.ctypes.data, xc.ctypes.data)
        return {"l_last": l_last, "beta": beta, "xc": xc}

    def set_state(self, l_last, beta, xc) -> None:
        l_last = np.ascontiguousarray(l_last, np.float32)
        beta = np.ascontiguousarray(beta, np.float32)
        xc = np.ascontiguousarray(xc, np.float32)
        esim_ad_set_state(self.ctx, l_last.ctypes.data, beta.ctypes.data, xc.ctypes.data)

    def reset(self) -> None:
        esim_ad_reset(self.ctx)
        self._keep.clear()
        self._t = 0

    def stats(self) -> dict:
        return esim_ad_stats_get(self.ctx)

    def profile(self, on: bool | None = None) -> dict | None:
        """profile(True) starts kernel timing (clearing it); profile() returns totals."""
        if on is not None:
            esim_ad_profile_enable(self.ctx, on)
            return None
        return esim_ad_profile_get(self.ctx)


# ------------------------------------------------------------- batching form

def esim_ad_batch_init(cfgs: list, cuda_stream: int = 0) -> int:
    arr = (esim_ad_config * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    _check(load_library().esim_ad_batch_init(arr, len(cfgs), ctypes.c_void_p(cuda_stream or None), ctypes.byref(h)),
           "esim_ad_batch_init")
    return h.value


def esim_ad_batch_step(b: int, frames: list) -> None:
    arr = (esim_ad_frame * len(frames))(*frames)
    _check(load_library().esim_ad_batch_step(ctypes.c_void_p(b), arr), "esim_ad_batch_step")


def esim_ad_batch_events(b: int, dst: int, cap: int, dst_is_device: bool = False) -> tuple[int, int]:
    n = ctypes.c_uint64(0)
    st = load_library().esim_ad_batch_events(ctypes.c_void_p(b), ctypes.c_void_p(dst or None), ctypes.c_uint64(cap),
                                             ctypes.byref(n), int(dst_is_device))
    return st, n.value


def esim_ad_batch_destroy(b: int) -> None:
    if b:
        load_library().esim_ad_batch_destroy(ctypes.c_void_p(b))


class Batch:
    """Many sequences stepped together (one config per sequence; width, height
    and contrast may differ).  ``step`` takes one frame dict per sequence (device
    tensors, as for Simulator.push) or None for a sequence idle this step."""

    def __init__(self, cfgs: list, stream=None):
        import torch
        self._torch = torch
        self.cfgs = cfgs
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.b = esim_ad_batch_init([c.c_config() for c in cfgs], self.stream.cuda_stream)
        self._keep = []

    def close(self):
        if getattr(self, "b", None):
            esim_ad_batch_destroy(self.b)
            self.b = None

    __del__ = close

    def step(self, frames: list) -> None:
        t = self._torch
        out = []
        for f in frames:
            if f is None:
                out.append(esim_ad_frame(None, None, None, None, None, None, 0, 0))
                continue
            for v in f.values():
                if not v.is_cuda or not v.is_contiguous():
                    raise ValueError("batched frames must be contiguous device tensors")
            g = lambda k: f[k].data_ptr() if k in f else None
            out.append(esim_ad_frame(g("radiance"), g("variance"), g("normal"), g("albedo"), g("depth"),
                                     g("features"), 0, 0))
            self._keep.append(f)
        esim_ad_batch_step(self.b, out)
        del t

    def events(self) -> np.ndarray:
        st, n = esim_ad_batch_events(self.b, 0, 0)
        if st not in (ESIM_AD_OK, ESIM_AD_ENOSPACE):
            raise EsimError(st, "esim_ad_batch_events")
        out = np.empty(n, BATCH_EVENT_DTYPE)
        if n:
            st, _ = esim_ad_batch_events(self.b, out.ctypes.data, n)
            _check(st, "esim_ad_batch_events")
        self._keep.clear()
        return out

    def events_device(self, dst, cap: int) -> int:
        st, n = esim_ad_batch_events(self.b, dst.data_ptr(), cap, dst_is_device=True)
        _check(st, "esim_ad_batch_events")
        self._keep.clear()
        return n

    def denoised(self, seq: int):
        t = self._torch
        c = self.cfgs[seq]
        a = t.empty(c.height, c.width, dtype=t.float32, device="cuda")
        f = t.empty(c.height, c.width, dtype=t.uint8, device="cuda")
        _check(load_library().esim_ad_batch_denoised(ctypes.c_void_p(self.b), seq, ctypes.c_void_p(a.data_ptr()),
                                                     ctypes.c_void_p(f.data_ptr()), 1), "esim_ad_batch_denoised")
        return a, f

    def get_state(self, seq: int) -> dict:
        c = self.cfgs[seq]
        n = c.width * c.height
        l_last, beta, xc = np.empty(n, np.float32), np.empty((n, 7), np.float32), np.empty((n, 7), np.float32)
        _check(load_library().esim_ad_batch_get_state(ctypes.c_void_p(self.b), seq, ctypes.c_void_p(l_last.ctypes.data),
                                                      ctypes.c_void_p(beta.ctypes.data), ctypes.c_void_p(xc.ctypes.data)),
               "esim_ad_batch_get_state")
        return {"l_last": l_last, "beta": beta, "xc": xc}

    def reset_sequence(self, seq: int) -> None:
        _check(load_library().esim_ad_batch_reset_sequence(ctypes.c_void_p(self.b), seq), "esim_ad_batch_reset_sequence")

    def stats(self) -> dict:
        s = esim_ad_stats()
        lanes = ctypes.c_int32(0)
        _check(load_library().esim_ad_batch_stats(ctypes.c_void_p(self.b), ctypes.byref(s), ctypes.byref(lanes)),
               "esim_ad_batch_stats")
        tw, th, ln = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load_library().esim_ad_batch_tiling(ctypes.c_void_p(self.b), ctypes.byref(tw), ctypes.byref(th),
                                                   ctypes.byref(ln)), "esim_ad_batch_tiling")
        return {"steps": s.frames, "regressions": s.regressions, "events": s.events, "pixels": s.pixels,
                "fp64_solves": s.fp64_solves, "lanes": lanes.value, "tile": (tw.value, th.value)}

    def profile(self, on: bool | None = None):
        lib = load_library()
        if on is not None:
            _check(lib.esim_ad_batch_profile_enable(ctypes.c_void_p(self.b), int(on)), "esim_ad_batch_profile_enable")
            return None
        p = esim_ad_profile()
        _check(lib.esim_ad_batch_profile_get(ctypes.c_void_p(self.b), ctypes.byref(p)), "esim_ad_batch_profile_get")
        return {"launches": {k: int(p.launches[i]) for i, k in enumerate(KERNEL_CLASSES)},
                "ms": {k: float(p.ms[i]) for i, k in enumerate(KERNEL_CLASSES)},
                "kernels": int(p.kernels), "neighbours": int(p.neighbours), "regressions": int(p.regressions)}
