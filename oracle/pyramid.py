"""Image pyramid of the photometric term (Sec. 3.4, dense photometric
alignment): a 3-level pyramid of the input image, each level Gaussian
blurred (kernel sizes 15, 9 and 3 from the coarsest to the finest level),
one Gauss-Newton iteration per level.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings (the paper gives the level count and the kernel sizes only):

* Level j = 0, 1, 2 (coarse to fine) has the downsampling factor
  d_j = 4, 2, 1: its pixel (x, y) is the mean of the full-resolution pixels
  of the d x d block [d x, d x + d) x [d y, d y + d) that lie in the image,
  so level j is ceil(W / d) x ceil(H / d), and its pixel centre sits at
  full-resolution coordinate d x + (d - 1) / 2.  A full-resolution
  projection u maps to u_j = (u - (d - 1) / 2) / d.
* The level is then blurred by a separable Gaussian of k taps (k odd),
  horizontal pass first, clamp to edge, with the usual size-to-width rule
  sigma = 0.3 ((k - 1) / 2 - 1) + 0.8 and taps exp(-i^2 / (2 sigma^2)),
  i = -(k-1)/2 .. (k-1)/2, normalised to sum 1 (k = 1: no blur).
* With L levels (1 <= L <= 3) the Gauss-Newton iteration g samples level
  j = min(3 - L + g, 2): L = 3 gives one iteration on each level and keeps
  the finest for any further iterations; the energy after the last update
  is taken on the finest level.  L = 0 keeps the raw image (no pyramid).
* Only the photometric term samples the pyramid; the silhouette term keeps
  the full-resolution distance transform.  Sampling at a level is the same
  bilinear clamp-to-edge sampling of the level image and of its central
  differences, the gradient scaled by 1 / d to full-resolution pixels.
"""
from __future__ import annotations

import numpy as np

FACTORS = (4, 2, 1)
DEFAULT_KSIZE = (15, 9, 3)


def gaussian_taps(k: int) -> np.ndarray:
    """Normalised Gaussian taps of an odd kernel size k (FP64)."""
    if k < 1 or k % 2 == 0:
        raise ValueError("kernel size must be odd and positive")
    r = (k - 1) // 2
    if r == 0:
        return np.ones(1)
    sigma = 0.3 * (r - 1) + 0.8
    i = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-i * i / (2.0 * sigma * sigma))
    return w / w.sum()


def box_downsample(img: np.ndarray, d: int) -> np.ndarray:
    """Mean over each d x d block (the part inside the image)."""
    img = np.asarray(img, dtype=np.float64)
    if d == 1:
        return img.copy()
    H, W = img.shape[:2]
    Hd, Wd = -(-H // d), -(-W // d)
    tail = img.shape[2:]
    s = np.zeros((Hd * d, Wd * d) + tail)
    c = np.zeros((Hd * d, Wd * d))
    s[:H, :W] = img
    c[:H, :W] = 1.0
    s = s.reshape((Hd, d, Wd, d) + tail).sum(axis=(1, 3))
    c = c.reshape(Hd, d, Wd, d).sum(axis=(1, 3))
    return s / c.reshape(c.shape + (1,) * len(tail))


def box_downsample_brute(img: np.ndarray, d: int) -> np.ndarray:
    """The same, one block at a time (small images)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape[:2]
    Hd, Wd = -(-H // d), -(-W // d)
    out = np.zeros((Hd, Wd) + img.shape[2:])
    for y in range(Hd):
        for x in range(Wd):
            out[y, x] = img[d * y:min(H, d * y + d), d * x:min(W, d * x + d)].mean(axis=(0, 1))
    return out


def blur(img: np.ndarray, k: int) -> np.ndarray:
    """Separable Gaussian blur with clamp to edge, rows first."""
    w = gaussian_taps(k)
    r = len(w) // 2
    img = np.asarray(img, dtype=np.float64)
    if r == 0:
        return img.copy()
    H, W = img.shape[:2]
    xs = np.arange(W)
    ys = np.arange(H)
    tmp = np.zeros_like(img)
    for i in range(-r, r + 1):
        tmp += w[i + r] * img[:, np.clip(xs + i, 0, W - 1)]
    out = np.zeros_like(img)
    for i in range(-r, r + 1):
        out += w[i + r] * tmp[np.clip(ys + i, 0, H - 1)]
    return out


def level_image(rgb: np.ndarray, j: int, ksize=DEFAULT_KSIZE) -> np.ndarray:
    """Level j (0 coarsest) of the pyramid of an RGB image."""
    return blur(box_downsample(rgb, FACTORS[j]), int(ksize[j]))


def level_of(gn: int, levels: int):
    """Pyramid level sampled at Gauss-Newton iteration gn (None: raw image)."""
    if levels <= 0:
        return None
    return min(3 - levels + gn, 2)


def to_level(u: np.ndarray, j: int) -> np.ndarray:
    """Full-resolution pixel coordinate -> level-j coordinate."""
    d = FACTORS[j]
    return (np.asarray(u, dtype=np.float64) - 0.5 * (d - 1)) / d
