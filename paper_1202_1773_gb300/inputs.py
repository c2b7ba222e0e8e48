"""Seeded synthetic "cartoon" images: the workloads the transform is tested and timed on.

Piecewise-constant shapes (filled ellipses and convex polygons with uniform
random intensities) on a zero background plus white Gaussian noise, the kind
of image the shearlet transform is built for (edges along curves).  The paper
uses no public dataset; these generators stand in for its test images.

This module holds none of the transform's arithmetic: both the CUDA path and
the FP64 oracle are fed from it in the tests and the benchmark.

Recipe (painted in order, later shapes overwrite earlier ones):
* ellipse: centre uniform over the image, semi-axes U[a_lo, a_hi] px,
  rotation U[0, pi), intensity U[0, 1];
* convex polygon: 3..8 vertices at sorted random angles on a circle of
  radius U[r_lo, r_hi] px around a uniform centre, intensity U[0, 1];
* noise N(0, sigma^2) added at the end, values not clipped.
All draws come from ``numpy.random.default_rng(seed)``.
"""

from __future__ import annotations

import numpy as np


def _paint_ellipse(img, rng, a_lo, a_hi):
    M, N = img.shape
    cy, cx = rng.uniform(0, M), rng.uniform(0, N)
    a, b = rng.uniform(a_lo, a_hi, size=2)
    th = rng.uniform(0.0, np.pi)
    val = rng.uniform(0.0, 1.0)
    y0, y1 = int(max(0, np.floor(cy - max(a, b)))), int(min(M, np.ceil(cy + max(a, b)) + 1))
    x0, x1 = int(max(0, np.floor(cx - max(a, b)))), int(min(N, np.ceil(cx + max(a, b)) + 1))
    if y0 >= y1 or x0 >= x1:
        return
    yy, xx = np.mgrid[y0:y1, x0:x1]
    dy, dx = yy - cy, xx - cx
    c, s = np.cos(th), np.sin(th)
    u = c * dx + s * dy
    w = -s * dx + c * dy
    inside = (u / a) ** 2 + (w / b) ** 2 <= 1.0
    img[y0:y1, x0:x1][inside] = val


def _paint_polygon(img, rng, r_lo, r_hi):
    M, N = img.shape
    cy, cx = rng.uniform(0, M), rng.uniform(0, N)
    nv = int(rng.integers(3, 9))
    r = rng.uniform(r_lo, r_hi)
    ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, nv))
    val = rng.uniform(0.0, 1.0)
    py = cy + r * np.sin(ang)
    px = cx + r * np.cos(ang)
    y0, y1 = int(max(0, np.floor(py.min()))), int(min(M, np.ceil(py.max()) + 1))
    x0, x1 = int(max(0, np.floor(px.min()))), int(min(N, np.ceil(px.max()) + 1))
    if y0 >= y1 or x0 >= x1:
        return
    yy, xx = np.mgrid[y0:y1, x0:x1]
    inside = np.ones(yy.shape, dtype=bool)
    for q in range(nv):
        ay, ax = py[q], px[q]
        by, bx = py[(q + 1) % nv], px[(q + 1) % nv]
        # counter-clockwise vertex order: interior on the left of each edge
        inside &= (bx - ax) * (yy - ay) - (by - ay) * (xx - ax) >= 0.0
    img[y0:y1, x0:x1][inside] = val


def cartoon(rows: int, cols: int, seed: int, n_ellipses: int, n_polygons: int = 0,
            size=(4.0, 20.0), sigma: float = 0.05, dtype=np.float64) -> np.ndarray:
    """One seeded cartoon image of shape (rows, cols)."""
    rng = np.random.default_rng(seed)
    img = np.zeros((rows, cols), dtype=np.float64)
    kinds = [0] * n_ellipses + [1] * n_polygons
    order = rng.permutation(len(kinds))
    for idx in order:
        if kinds[idx] == 0:
            _paint_ellipse(img, rng, size[0], size[1])
        else:
            _paint_polygon(img, rng, size[0], size[1])
    img += rng.normal(0.0, sigma, size=img.shape)
    return img.astype(dtype)


def small_cartoon(seed: int = 0) -> np.ndarray:
    """64x64 float64: 6 ellipses (semi-axes 4-20 px) + N(0, 0.05^2)."""
    return cartoon(64, 64, seed, n_ellipses=6, size=(4.0, 20.0), sigma=0.05, dtype=np.float64)


def medium_cartoon(seed: int = 1, rows: int = 512, cols: int = 512) -> np.ndarray:
    """512x512 float32: 20 ellipses + 20 convex polygons (8-64 px) + N(0, 0.1^2)."""
    return cartoon(rows, cols, seed, n_ellipses=20, n_polygons=20, size=(8.0, 64.0),
                   sigma=0.1, dtype=np.float32)


def scaled_cartoon(rows: int, cols: int, seed: int, sigma: float = 0.1) -> np.ndarray:
    """float32 cartoon with a shape count proportional to the area (at least 6).

    40 shapes per 512x512, half ellipses and half polygons, sizes 8-64 px.
    """
    n = max(6, int(round(40 * rows * cols / (512 * 512))))
    return cartoon(rows, cols, seed, n_ellipses=(n + 1) // 2, n_polygons=n // 2,
                   size=(8.0, 64.0), sigma=sigma, dtype=np.float32)


def noise_image(rows: int, cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Uniform U[0,1) random image (the paper's "random image" of Sec. 3.6)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, (rows, cols)).astype(dtype)


def batch_sizes(n_images: int, seed: int = 2):
    """Uneven (rows, cols) mix for the batched workload, drawn uniformly from
    {128^2, 256^2, 480x640, 512^2, 768x1024, 1024^2}."""
    choices = [(128, 128), (256, 256), (480, 640), (512, 512), (768, 1024), (1024, 1024)]
    rng = np.random.default_rng(seed)
    return [choices[int(q)] for q in rng.integers(0, len(choices), n_images)]
