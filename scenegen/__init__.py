"""Seeded synthetic inputs shared by the oracle and the CUDA path (no method arithmetic)."""
from .scene import SceneConfig, config, make_scene, noise_free, counts, window_config, KINDS, MEAS_DIM  # noqa: F401
