"""Body-part mask of the silhouette term (Sec. 3.4, dense silhouette
alignment): the posed model V^S is projected into the frame, a body-part
label image is formed from the skinning weights, each part is grown by a
dilation of at most 10 pixels with the torso taking precedence, and a
contour vertex whose projection lands on a region of another part has its
silhouette term switched off (b_i = 0).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings (the paper names the ingredients only):

* A vertex's part is the part of the bone with its largest skinning weight
  (the first of equal weights), through a bone -> part table.
* The label image comes from the z-buffer of V^S (the exact rasteriser of
  module ``visibility``): a covered pixel takes the label of its front
  triangle, which is the label two or three of its vertices share, else its
  first vertex's label.  Uncovered pixels have no label (NONE = 255).
* Dilation: an unlabelled pixel within Euclidean distance R (pixel centres,
  d^2 <= R^2) of labelled pixels takes the torso label if a torso pixel is
  among them, else the label of the nearest one (the lower label on equal
  distances); labelled pixels keep their label.
* At each linearisation a contour vertex with projection (u, v) reads the
  label at pixel (floor(u + 1/2), floor(v + 1/2)), decided in FP32 (the
  kernel's precision: positions rounded to FP32, the projection's operations
  each rounded once); a label other than NONE and other than the vertex's
  part switches its silhouette residual off.
"""
from __future__ import annotations

import numpy as np

NONE = 255


def vertex_parts(skin_idx: np.ndarray, skin_w: np.ndarray, bone_part: np.ndarray) -> np.ndarray:
    """(N,) uint8 part of every vertex: the part of its heaviest bone."""
    w = np.asarray(skin_w, dtype=np.float32)
    s = np.argmax(w, axis=1)                      # the first maximum
    bone = np.asarray(skin_idx)[np.arange(len(w)), s]
    return np.asarray(bone_part, dtype=np.int64)[bone].astype(np.uint8)


def triangle_labels(F: np.ndarray, vpart: np.ndarray) -> np.ndarray:
    """Label of every triangle: the label shared by two or three of its
    vertices, else its first vertex's."""
    a, b, c = (vpart[np.asarray(F)[:, k]] for k in range(3))
    return np.where((a == b) | (a == c), a, np.where(b == c, b, a)).astype(np.uint8)


def label_image(zbuf: np.ndarray, F: np.ndarray, vpart: np.ndarray) -> np.ndarray:
    """(H,W) uint8 label of the front triangle of each pixel (NONE: empty)."""
    empty = zbuf == np.uint64(0xFFFFFFFFFFFFFFFF)
    tri = (zbuf & np.uint64(0xFFFFFFFF)).astype(np.int64)
    lab = triangle_labels(F, vpart)
    out = np.full(zbuf.shape, NONE, dtype=np.uint8)
    out[~empty] = lab[tri[~empty]]
    return out


def dilate(raw: np.ndarray, radius: int, torso: int) -> np.ndarray:
    """Grow every part into unlabelled pixels within ``radius`` (see the
    module docstring); torso < 0: no part has precedence."""
    raw = np.asarray(raw, dtype=np.uint8)
    H, W = raw.shape
    big = np.iinfo(np.int64).max
    best_d = np.full((H, W), big, dtype=np.int64)
    best_l = np.full((H, W), NONE, dtype=np.int64)
    torso_near = np.zeros((H, W), dtype=bool)
    R = int(radius)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            d2 = dy * dy + dx * dx
            if d2 > R * R:
                continue
            # label of pixel (y + dy, x + dx), NONE outside the image
            src = np.full((H, W), NONE, dtype=np.int64)
            ys0, ys1 = max(0, -dy), min(H, H - dy)
            xs0, xs1 = max(0, -dx), min(W, W - dx)
            if ys0 < ys1 and xs0 < xs1:
                src[ys0:ys1, xs0:xs1] = raw[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
            has = src != NONE
            torso_near |= has & (src == torso)
            better = has & ((d2 < best_d) | ((d2 == best_d) & (src < best_l)))
            best_d = np.where(better, d2, best_d)
            best_l = np.where(better, src, best_l)
    grown = np.where(torso_near, torso, best_l)
    return np.where(raw != NONE, raw, grown).astype(np.uint8)


def dilate_brute(raw: np.ndarray, radius: int, torso: int) -> np.ndarray:
    """The same, pixel by pixel over every labelled pixel (small images)."""
    raw = np.asarray(raw, dtype=np.uint8)
    H, W = raw.shape
    ys, xs = np.nonzero(raw != NONE)
    out = raw.copy()
    for y in range(H):
        for x in range(W):
            if raw[y, x] != NONE or len(ys) == 0:
                continue
            d2 = (ys - y) ** 2 + (xs - x) ** 2
            near = d2 <= radius * radius
            if not near.any():
                continue
            labs = raw[ys[near], xs[near]].astype(np.int64)
            if torso >= 0 and (labs == torso).any():
                out[y, x] = torso
                continue
            dn = d2[near]
            m = dn == dn.min()
            out[y, x] = labs[m].min()
    return out


def part_mask(V32: np.ndarray, F: np.ndarray, f, cx, cy, W, H, vpart, radius=10, torso=0) -> np.ndarray:
    """The frame's part mask from the FP32 posed model V^S."""
    from . import visibility as _vis
    out = _vis.visibility(np.asarray(V32, dtype=np.float32), F, f, cx, cy, W, H,
                          np.zeros((H, W), np.float32), np.zeros((H, W), np.uint8))
    return dilate(label_image(out["zbuf"], F, vpart), radius, torso)


def masked(P, V: np.ndarray) -> np.ndarray:
    """Vertices at positions V (N,3) whose silhouette term is switched off:
    the label at the pixel of their projection differs from their part.  The
    pixel is decided in FP32 like the kernel: the positions rounded to FP32,
    u = (f X) / Z + cx with every operation rounded once, then
    floor(u + 1/2)."""
    N = len(V)
    if getattr(P, "part_mask", None) is None:
        return np.zeros(N, dtype=bool)
    H, W = P.part_mask.shape
    V32 = np.asarray(V, dtype=np.float32)
    f, cx, cy, half = np.float32(P.f), np.float32(P.cx), np.float32(P.cy), np.float32(0.5)
    ok = V32[:, 2] > np.float32(1e-3)
    Z = np.where(ok, V32[:, 2], np.float32(1.0))
    u = (f * V32[:, 0]) / Z + cx
    v = (f * V32[:, 1]) / Z + cy
    px = np.floor(u + half)
    py = np.floor(v + half)
    ok &= (px >= 0) & (px < W) & (py >= 0) & (py < H)
    lab = np.full(N, NONE, dtype=np.int64)
    lab[ok] = P.part_mask[py[ok].astype(np.int64), px[ok].astype(np.int64)]
    return (lab != NONE) & (lab != np.asarray(P.vpart, dtype=np.int64))
