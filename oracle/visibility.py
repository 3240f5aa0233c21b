"""Loader for the exact-arithmetic visibility oracle (``visibility.c``).

TEST INFRASTRUCTURE ONLY.  ``build()`` compiles the C file with gcc into
``oracle/_build/`` (no contraction of FP32 operations); ``visibility()``
calls it.  ``mesh_edges()`` is the oracle's own mesh-edge adjacency.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "visibility.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_visibility.so")
_lib = None

FLAG_VISIBLE, FLAG_ONSIL, FLAG_INB, FLAG_BNEG = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile visibility.c (gcc, -ffp-contract=off) if missing or stale."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.oracle_visibility.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int,
                                           ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_int, ctypes.c_int, P, P, ctypes.c_float, P, P, P]
        _lib.oracle_visibility.restype = None
        _lib.oracle_directions.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_float, ctypes.c_int, ctypes.c_int, P, P, P, P]
        _lib.oracle_directions.restype = None
    return _lib


def mesh_edges(F: np.ndarray) -> np.ndarray:
    """Undirected mesh edges (v0 < v1) with their triangles: (NE, 4) int32
    rows (v0, v1, t0, t1), t0 < t1, t1 = -1 for a boundary edge; sorted by
    (v0, v1).  Raises on a non-manifold edge (more than two triangles)."""
    F = np.asarray(F, dtype=np.int64)
    T = len(F)
    a = np.concatenate([F[:, 0], F[:, 1], F[:, 2]])
    b = np.concatenate([F[:, 1], F[:, 2], F[:, 0]])
    t = np.tile(np.arange(T), 3)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    o = np.lexsort((t, hi, lo))
    lo, hi, t = lo[o], hi[o], t[o]
    rows = []
    i = 0
    n = len(lo)
    while i < n:
        j = i
        while j < n and lo[j] == lo[i] and hi[j] == hi[i]:
            j += 1
        if j - i > 2:
            raise ValueError("non-manifold mesh edge")
        rows.append((lo[i], hi[i], t[i], t[i + 1] if j - i == 2 else -1))
        i = j
    return np.asarray(rows, dtype=np.int32).reshape(-1, 4)


def visibility(Vwarp32, F, cam_f, cam_cx, cam_cy, W, H, DT, mask, eps=1e-2, edges=None):
    """Run the exact decisions on FP32 warped positions.

    Returns dict(uv (N,2) f32, zbuf (H,W) uint64, flags (N,) uint8).
    """
    lib = _load()
    V = np.ascontiguousarray(Vwarp32, dtype=np.float32)
    Fi = np.ascontiguousarray(F, dtype=np.int32)
    E = mesh_edges(Fi) if edges is None else np.ascontiguousarray(edges, dtype=np.int32)
    D = np.ascontiguousarray(DT, dtype=np.float32)
    M = np.ascontiguousarray(mask, dtype=np.uint8)
    assert D.shape == (H, W) and M.shape == (H, W)
    N = len(V)
    uv = np.zeros((N, 2), dtype=np.float32)
    zbuf = np.zeros((H, W), dtype=np.uint64)
    flags = np.zeros(N, dtype=np.uint8)
    lib.oracle_visibility(V.ctypes.data, N, Fi.ctypes.data, len(Fi), E.ctypes.data, len(E),
                          float(np.float32(cam_f)), float(np.float32(cam_cx)),
                          float(np.float32(cam_cy)), int(W), int(H), D.ctypes.data,
                          M.ctypes.data, float(np.float32(eps)), uv.ctypes.data, zbuf.ctypes.data,
                          flags.ctypes.data)
    return dict(uv=uv, zbuf=zbuf, flags=flags)


def directions(Vwarp32, F, cam_f, cam_cx, cam_cy, W, H, DT, mask, sel):
    """b_i = -1 flags (bool) of the selected vertices at the FP32 surface
    Vwarp32 (the direction rule re-evaluated on the current surface)."""
    lib = _load()
    V = np.ascontiguousarray(Vwarp32, dtype=np.float32)
    Fi = np.ascontiguousarray(F, dtype=np.int32)
    D = np.ascontiguousarray(DT, dtype=np.float32)
    M = np.ascontiguousarray(mask, dtype=np.uint8)
    S = np.ascontiguousarray(sel, dtype=np.uint8)
    out = np.zeros(len(V), dtype=np.uint8)
    lib.oracle_directions(V.ctypes.data, len(V), Fi.ctypes.data, len(Fi), float(np.float32(cam_f)),
                          float(np.float32(cam_cx)), float(np.float32(cam_cy)), int(W), int(H), D.ctypes.data,
                          M.ctypes.data, S.ctypes.data, out.ctypes.data)
    return out != 0
