"""Silhouette distance transform (Sec. 3.2: distance transform images from
the foreground silhouettes), exactly.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading (the paper gives no definition): the contour pixels are the
foreground pixels with a 4-neighbour in the background or on the image
border; I_DT at a pixel is the Euclidean distance, in pixels, between pixel
centres to the nearest contour pixel (0 on the contour).  Without any contour
pixel (an empty silhouette) I_DT is 0 everywhere.  The squared distances are
integers; the distance is their square root rounded once to FP32, the
precision the solver samples it in.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def contour(mask: np.ndarray) -> np.ndarray:
    """Contour pixels of a silhouette (bool H x W)."""
    m = np.asarray(mask, dtype=bool)
    pad = np.pad(m, 1, constant_values=False)
    interior = pad[1:-1, 1:-1] & pad[:-2, 1:-1] & pad[2:, 1:-1] & pad[1:-1, :-2] & pad[1:-1, 2:]
    return m & ~interior


def squared_edt(mask: np.ndarray) -> np.ndarray:
    """Integer squared distance to the nearest contour pixel (int64; -1 where
    the silhouette has no contour), by SciPy's exact Euclidean transform."""
    c = contour(mask)
    if not c.any():
        return np.full(c.shape, -1, dtype=np.int64)
    d = ndimage.distance_transform_edt(~c)
    return np.rint(d * d).astype(np.int64)


def squared_edt_brute(mask: np.ndarray) -> np.ndarray:
    """The same by brute force over all contour pixels (small masks)."""
    c = contour(mask)
    H, W = c.shape
    ys, xs = np.nonzero(c)
    if len(ys) == 0:
        return np.full((H, W), -1, dtype=np.int64)
    yy, xx = np.mgrid[:H, :W]
    d2 = (yy[..., None] - ys) ** 2 + (xx[..., None] - xs) ** 2
    return d2.min(-1).astype(np.int64)


def distance_transform(mask: np.ndarray) -> np.ndarray:
    """I_DT in FP32: sqrt of the integer squared distance, rounded once."""
    d2 = squared_edt(mask)
    out = np.sqrt(np.maximum(d2, 0).astype(np.float32))
    return np.where(d2 < 0, np.float32(0.0), out).astype(np.float32)
