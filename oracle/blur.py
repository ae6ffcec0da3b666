"""Adaptive Gaussian blur oracle — TEST INFRASTRUCTURE ONLY.

Sec. 2.2: an image post-process whose filter size follows the local image
resolution.  Reading (the same as the library's): the local resolution of a
pixel is the density-weighted mean leaf level of its ray; sigma (pixels) =
2^-level / (2 pixel); below half a pixel the pixel is copied; otherwise a row
pass then a column pass, each output pixel gathering with its own sigma,
weights exp(-k^2 / (2 sigma^2)) for |k| <= floor(3 sigma + 0.5) (at most 64),
renormalised over the samples inside the map.  Plain float64 loops.
"""
from __future__ import annotations

import math

import numpy as np

MAX_RADIUS = 64


def sigma_map(level: np.ndarray, pixel: float) -> np.ndarray:
    return 0.5 * np.exp2(-np.asarray(level, np.float64)) / pixel


def _pass(img: np.ndarray, sig: np.ndarray, axis: int) -> np.ndarray:
    ny, nx = img.shape
    out = np.empty_like(img, dtype=np.float64)
    for y in range(ny):
        for x in range(nx):
            s = sig[y, x]
            if not s >= 0.5:
                out[y, x] = img[y, x]
                continue
            R = min(MAX_RADIUS, int(3.0 * s + 0.5))
            acc = norm = 0.0
            for k in range(-R, R + 1):
                xx, yy = (x + k, y) if axis == 1 else (x, y + k)
                if 0 <= xx < nx and 0 <= yy < ny:
                    w = math.exp(-k * k / (2.0 * s * s))
                    acc += w * img[yy, xx]
                    norm += w
            out[y, x] = acc / norm
    return out


def adaptive_blur(img: np.ndarray, level: np.ndarray, pixel: float) -> np.ndarray:
    sig = sigma_map(level, pixel)
    return _pass(_pass(np.asarray(img, np.float64), sig, axis=1), sig, axis=0)
