"""Seeded synthetic Gaussian scenes and cameras.

This package only draws random inputs. It holds none of the rasterizer's
arithmetic (no projection, no compositing, no gradients), so both the
FP64 oracle and the CUDA path can consume the same inputs without sharing
any of the method's code.
"""
from .generate import (  # noqa: F401
    Scene,
    camera_array,
    look_at,
    make_scene,
    perturb_pose,
    random_image,
    sh_coefficients,
    SCENE_CONFIGS,
)
