"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package produces inputs only: camera intrinsics, camera trajectories,
analytic ray-cast renders (intensity, ground-truth depth, surface normals),
and photometric noise. It holds none of the tracking method's arithmetic (no
warp function, no factors, no belief propagation). Rotations come from scipy.
"""
from .scenes import (Camera, Scene, Plane, HeightField, BlockTexture,
                     SmoothTexture, render)
from .sequences import (Sequence, tiny_pair, scamp_room, realistic,
                        batched_family, adjoint_family, affine_pair,
                        ppa_noise, THETA_STRONG, THETA_MILD)

__all__ = [
    "Camera", "Scene", "Plane", "HeightField", "BlockTexture", "SmoothTexture",
    "render", "Sequence", "tiny_pair", "scamp_room", "realistic",
    "batched_family", "adjoint_family", "affine_pair", "ppa_noise",
    "THETA_STRONG", "THETA_MILD",
]
