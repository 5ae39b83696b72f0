"""Seeded synthetic bundle-adjustment scenes.

This package only draws random inputs (cameras on a circle, points in a cube,
visibility, pixel noise, outliers, perturbed initial estimates). It holds no
residual, Jacobian, linear-system or solver arithmetic, so the CPU oracle and
the CUDA path can both consume its output without sharing any of the method.
"""
from .generate import (  # noqa: F401
    Scene,
    make_scene,
    config_scene,
    make_windows,
    CONFIGS,
)
