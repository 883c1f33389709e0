"""Seeded synthetic stand-ins for the paper's 8-bit greyscale test images.

The paper measures on two 512x512 photographs (Section 4) that are not
available here.  These generators draw images with the same size, bit depth
and the mix of smooth regions, texture and noise that drives the quadtree:

* ``gaussian_scene(N, seed)``: 12 Gaussian blobs (centre U[0,N)^2,
  amplitude U[40,200], sigma U[8,48] px) + a linear gradient (random angle,
  0 -> U[0,64] across the image) + 4 sinusoidal texture patches (square side
  U[N/8,N/4], period U[4,16] px, random orientation, amplitude U[10,40]) +
  N(0,6) noise, rounded and clipped to [0,255].
* ``voronoi(N, seed)``: 64 seeds U[0,N)^2, integer grey levels U[0,255],
  nearest seed by squared distance, ties to the lowest seed index.

Every draw comes from ``numpy.random.default_rng(seed)`` in a fixed order, so
an image is a pure function of (N, seed).  Nothing here computes any part of
the fractal coder.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gaussian_scene", "voronoi", "constant", "scene256_image", "scenes512_images",
    "exhaustive_images", "mixed_sides", "mixed_images", "serving_requests",
]


def gaussian_scene(N: int, seed: int, H: int | None = None) -> np.ndarray:
    """Blobs + gradient + sinusoid patches + noise, uint8 of shape (H, N)."""
    W = int(N)
    H = W if H is None else int(H)
    rng = np.random.default_rng(seed)
    xs = np.arange(W, dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)
    img = np.zeros((H, W), dtype=np.float64)
    side = min(W, H)
    for _ in range(12):
        cx = rng.uniform(0, W)
        cy = rng.uniform(0, H)
        amp = rng.uniform(40, 200)
        sig = rng.uniform(8, 48)
        gx = np.exp(-((xs - cx) ** 2) / (2 * sig * sig))
        gy = np.exp(-((ys - cy) ** 2) / (2 * sig * sig))
        img += amp * np.outer(gy, gx)
    ang = rng.uniform(0, 2 * math.pi)
    gamp = rng.uniform(0, 64)
    proj = np.cos(ang) * xs[None, :] + np.sin(ang) * ys[:, None]
    lo, hi = proj.min(), proj.max()
    img += gamp * (proj - lo) / max(hi - lo, 1e-9)
    for _ in range(4):
        ps = int(rng.uniform(side / 8, side / 4))
        px = int(rng.uniform(0, W - ps))
        py = int(rng.uniform(0, H - ps))
        period = rng.uniform(4, 16)
        theta = rng.uniform(0, math.pi)
        pamp = rng.uniform(10, 40)
        lx = xs[px:px + ps][None, :]
        ly = ys[py:py + ps][:, None]
        img[py:py + ps, px:px + ps] += pamp * np.sin(
            2 * math.pi * (lx * math.cos(theta) + ly * math.sin(theta)) / period)
    img += rng.normal(0.0, 6.0, size=(H, W))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def voronoi(N: int, seed: int, H: int | None = None, cells: int = 64) -> np.ndarray:
    """Piecewise-constant image: nearest of ``cells`` random seeds."""
    W = int(N)
    H = W if H is None else int(H)
    rng = np.random.default_rng(seed)
    sx = rng.uniform(0, W, size=cells)
    sy = rng.uniform(0, H, size=cells)
    grey = rng.integers(0, 256, size=cells)
    out = np.empty((H, W), dtype=np.uint8)
    xs = np.arange(W, dtype=np.float64)
    for y in range(H):
        d2 = (xs[None, :] - sx[:, None]) ** 2 + (y - sy[:, None]) ** 2
        out[y] = grey[np.argmin(d2, axis=0)]
    return out


def constant(N: int, value: int, H: int | None = None) -> np.ndarray:
    H = N if H is None else H
    return np.full((H, N), value, dtype=np.uint8)


# ---- workload recipes (one per measured configuration) -------------------

def scene256_image() -> np.ndarray:
    """256x256 scene, seed 0 (MNS 16->8->4, RMS threshold 8, decode 10 its)."""
    return gaussian_scene(256, 0)


def scenes512_images() -> list[tuple[str, np.ndarray]]:
    """512x512: scenes with seeds 1..8 and Voronoi images with seeds 101, 102."""
    out = [(f"scene{s}", gaussian_scene(512, s)) for s in range(1, 9)]
    out += [(f"voronoi{s}", voronoi(512, s)) for s in (101, 102)]
    return out


def exhaustive_images() -> list[tuple[str, np.ndarray]]:
    """Exhaustive-search workloads: 512x512 seed 1 and 1024x1024 seed 9."""
    return [("scene1_512", gaussian_scene(512, 1)), ("scene9_1024", gaussian_scene(1024, 9))]


def mixed_sides(count: int = 512) -> np.ndarray:
    """Mixed sides {256,512,1024,2048} with weights .4/.3/.2/.1 from rng(4)."""
    rng = np.random.default_rng(4)
    return rng.choice(np.array([256, 512, 1024, 2048]), size=count, p=[0.4, 0.3, 0.2, 0.1])


def mixed_images(count: int = 512):
    """Yield (index, image) for the mixed-size batch; image i uses seed 1000+i."""
    for i, s in enumerate(mixed_sides(count)):
        yield i, gaussian_scene(int(s), 1000 + i)


def serving_requests(rate: float = 2000.0, seconds: float = 60.0, encode_frac: float = 0.8):
    """Poisson arrival times, request kinds and sides for the serving workload.

    Returns arrays (t_arrival [s], is_encode [bool], side [px], seed).  Sides
    are log-uniform in [128, 4096] rounded to a multiple of 32; request i
    draws its image from seed 10**6 + i.
    """
    rng = np.random.default_rng(5)
    n_est = int(rate * seconds * 1.2) + 64
    gaps = rng.exponential(1.0 / rate, size=n_est)
    t = np.cumsum(gaps)
    t = t[t < seconds]
    n = t.size
    is_enc = rng.uniform(size=n) < encode_frac
    u = rng.uniform(math.log(128), math.log(4096), size=n)
    side = (32 * np.rint(np.exp(u) / 32)).astype(np.int64)
    side = np.clip(side, 128, 4096)
    seeds = 10 ** 6 + np.arange(n)
    return t, is_enc, side, seeds
