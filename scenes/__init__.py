"""Seeded synthetic input frames (radiance, variance, normal, albedo, depth).

Shared by the CUDA path's tests, the oracle's tests and the benchmark; holds
none of the method's arithmetic.
"""
from .generator import Scene, SceneConfig, batch_configs, preset, rect_layout  # noqa: F401
from .philox import philox4x32, uniform_open01  # noqa: F401
