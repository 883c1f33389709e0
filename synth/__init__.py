"""Seeded synthetic greyscale inputs shared by the oracle tests and the CUDA path.

This package holds no part of the fractal coding arithmetic: it only draws
images (and workload recipes) from numpy's PCG64 generator.  Both the oracle
and the GPU path consume the bytes it produces, so image generation is not
part of any parity check.
"""
from .images import (  # noqa: F401
    gaussian_scene,
    voronoi,
    constant,
    scene256_image,
    scenes512_images,
    exhaustive_images,
    mixed_sides,
    mixed_images,
    serving_requests,
)
