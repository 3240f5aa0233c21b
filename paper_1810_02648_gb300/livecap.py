"""Thin ctypes binding of the livecap C ABI (include/livecap.h).

Argument marshalling only: every computation runs in the CUDA library.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
device memory); they must be C-contiguous with the dtype the C call takes.
Outputs default to freshly allocated numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

LC_OK, LC_ERR_ARG, LC_ERR_STATE, LC_ERR_CUDA, LC_ERR_NUMERIC, LC_ERR_TIMEOUT, LC_ERR_OOM = 0, -1, -2, -3, -4, -5, -6
LC_MAX_GN = 64
FLAG_VISIBLE, FLAG_ONSIL, FLAG_INB, FLAG_BNEG, FLAG_PRUNED, FLAG_MASKED = 1, 2, 4, 8, 16, 32


class lc_params(ctypes.Structure):
    _fields_ = [("w_photo", ctypes.c_float), ("w_sil", ctypes.c_float), ("w_arap", ctypes.c_float),
                ("n_gn", ctypes.c_int), ("n_pcg", ctypes.c_int), ("eps_vis", ctypes.c_float),
                ("lambda_2d", ctypes.c_float), ("lambda_3d", ctypes.c_float), ("lambda_sil", ctypes.c_float),
                ("n_gn_pose", ctypes.c_int), ("lambda_prior", ctypes.c_float), ("pcg_kernel", ctypes.c_int),
                ("target_energy", ctypes.c_float), ("w_smooth", ctypes.c_float), ("w_edge", ctypes.c_float),
                ("w_velocity", ctypes.c_float), ("w_acceleration", ctypes.c_float),
                ("n_gn_surface", ctypes.c_int), ("n_pcg_surface", ctypes.c_int), ("pose_solver", ctypes.c_int),
                ("lambda_temporal", ctypes.c_float), ("lambda_anatomic", ctypes.c_float), ("sigma_c", ctypes.c_float),
                ("pyr_levels", ctypes.c_int), ("pyr_ksize", ctypes.c_int * 3), ("pose_displacement", ctypes.c_int),
                ("gn_block", ctypes.c_int),
                ("graph_warp", ctypes.c_int),
                ("tma_taps", ctypes.c_int)]


class lc_solve_stats(ctypes.Structure):
    _fields_ = [("e_photo", ctypes.c_double), ("e_sil", ctypes.c_double), ("e_arap", ctypes.c_double),
                ("e_total", ctypes.c_double), ("e_gn", ctypes.c_double * LC_MAX_GN),
                ("step_norm", ctypes.c_double * LC_MAX_GN), ("pcg_iters", ctypes.c_int * LC_MAX_GN),
                ("n_gn_done", ctypes.c_int), ("n_visible", ctypes.c_int), ("n_boundary", ctypes.c_int),
                ("n_boundary_neg", ctypes.c_int), ("pcg_breakdowns", ctypes.c_int),
                ("n_kernels", ctypes.c_int), ("pcg_cluster_size", ctypes.c_int),
                ("e_smooth", ctypes.c_double), ("e_edge", ctypes.c_double), ("e_velocity", ctypes.c_double),
                ("e_acceleration", ctypes.c_double), ("n_kernels_step", ctypes.c_int)]

    def to_dict(self) -> dict:
        g = self.n_gn_done
        return dict(e_photo=self.e_photo, e_sil=self.e_sil, e_arap=self.e_arap, e_total=self.e_total,
                    e_gn=list(self.e_gn[:g]), step_norm=list(self.step_norm[:g]),
                    pcg_iters=list(self.pcg_iters[:g]), n_visible=self.n_visible,
                    n_boundary=self.n_boundary, n_boundary_neg=self.n_boundary_neg,
                    pcg_breakdowns=self.pcg_breakdowns, n_kernels=self.n_kernels,
                    pcg_cluster_size=self.pcg_cluster_size, n_gn_done=g,
                    e_gn_all=list(self.e_gn), e_smooth=self.e_smooth, e_edge=self.e_edge,
                    e_velocity=self.e_velocity, e_acceleration=self.e_acceleration,
                    n_kernels_step=self.n_kernels_step)


_P = ctypes.c_void_p
_SIGS = {
    "lc_create": [ctypes.POINTER(_P), ctypes.c_int, _P],
    "lc_destroy": [_P],
    "lc_last_error": [_P],
    "lc_params_default": [ctypes.POINTER(lc_params)],
    "lc_set_params": [_P, ctypes.POINTER(lc_params)],
    "lc_set_camera": [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int],
    "lc_upload_template": [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P],
    "lc_build_graph": [_P, ctypes.c_int, ctypes.c_int],
    "lc_upload_graph": [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P],
    "lc_read_graph": [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int)],
    "lc_set_node_params": [_P, _P, _P],
    "lc_upload_frame": [_P, _P, _P, _P, _P, _P],
    "lc_solve_nonrigid": [_P, ctypes.POINTER(lc_solve_stats)],
    "lc_read_back": [_P, _P, _P, _P, _P, _P],
    "lc_compute_visibility": [_P],
    "lc_read_visibility": [_P, _P, _P, _P],
    "lc_eval_linearization": [_P, _P, _P, _P, _P, _P, _P, _P],
    "lc_eval_gradient": [_P, _P, _P],
    "lc_apply_jtj": [_P, _P, _P],
    "lc_solve_linear": [_P, _P, ctypes.POINTER(ctypes.c_int)],
    "lc_upload_skeleton": [_P, ctypes.c_int, _P, _P, _P, _P, _P],
    "lc_set_pose": [_P, _P],
    "lc_reset_pose": [_P],
    "lc_batch_create": [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int],
    "lc_batch_destroy": [_P],
    "lc_batch_last_error": [_P],
    "lc_batch_set_pcg_mode": [_P, ctypes.c_int],
    "lc_batch_solve": [_P, ctypes.c_int, ctypes.POINTER(lc_solve_stats)],
    "lc_batch_autotune": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _P],
    "lc_batch_stream": [_P],
    "lc_batch_apply_jtj": [_P, ctypes.c_int],
    "lc_batch_step": [_P, _P, ctypes.c_uint, _P],
    "lc_batch_set_shape": [_P, _P],
    "lc_batch_get_shape": [_P, _P],
    "lc_batch_autotune_shapes": [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)],
    "lc_batch_size_class": [_P, ctypes.c_char_p, ctypes.c_int],
    "lc_autotune_table": [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "lc_autotune_table_load": [ctypes.c_char_p],
    "lc_mlp_create": [ctypes.POINTER(_P), ctypes.c_int, _P, _P, _P],
    "lc_mlp_destroy": [_P],
    "lc_mlp_last_error": [_P],
    "lc_mlp_get_params": [_P, _P],
    "lc_mlp_set_scaling": [_P, _P, _P, _P],
    "lc_mlp_set_gemm": [_P, ctypes.c_int],
    "lc_mlp_get_scaling": [_P, _P, _P, _P],
    "lc_mlp_fit_scaling": [_P, _P, _P, ctypes.c_longlong],
    "lc_mlp_forward": [_P, _P, ctypes.c_int, _P],
    "lc_mlp_gradient": [_P, _P, _P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)],
    "lc_mlp_train_step": [_P, _P, _P, _P, ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_double)],
    "lc_node_features": [_P, _P],
    "lc_read_stats": [_P, ctypes.POINTER(lc_solve_stats)],
    "lc_record_motion": [_P],
    "lc_read_motion": [_P, _P],
    "lc_warm_start": [_P, _P, ctypes.POINTER(ctypes.c_int), _P],
    "lc_solve_pose": [_P, ctypes.POINTER(lc_solve_stats)],
    "lc_eval_pose": [_P, _P, _P, _P, _P],
    "lc_set_profiling": [_P, ctypes.c_int],
    "lc_read_profile": [_P, _P, _P],
    "lc_set_rest_geometry": [_P, _P],
    "lc_read_frame": [_P, _P, _P],
    "lc_set_body_parts": [_P, _P, ctypes.c_int, ctypes.c_int],
    "lc_read_part_mask": [_P, _P, _P],
    "lc_read_pyramid_level": [_P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "lc_set_pose_priors": [_P, _P, _P, _P],
    "lc_pose_advance": [_P],
    "lc_pose_extrapolate": [_P],
    "lc_pose_clear_history": [_P],
    "lc_set_surface": [_P, _P],
    "lc_surface_start": [_P],
    "lc_surface_history": [_P, _P, _P],
    "lc_surface_advance": [_P],
    "lc_solve_surface": [_P, ctypes.POINTER(lc_solve_stats)],
    "lc_read_surface": [_P, _P, _P],
    "lc_surface_visibility": [_P],
    "lc_surface_linearize": [_P, _P, _P, _P],
    "lc_surface_apply_jtj": [_P, _P, _P],
    "lc_surface_solve_linear": [_P, _P, ctypes.POINTER(ctypes.c_int)],
    "lc_visibility_noalloc": [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_int, ctypes.c_int, ctypes.c_float, _P, _P],
}
PHASES = ["warp", "visibility", "linearize", "rhs", "pcg_init", "jtj", "pcg_vec", "update", "pose", "pcg",
          "pose_vis", "pose_system", "pose_solve"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load liblivecap.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"livecap library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("lc_last_error", "lc_batch_last_error", "lc_mlp_last_error") \
            else ctypes.c_int
        if name == "lc_batch_stream":
            fn.restype = _P
    _lib = lib
    return lib


class LivecapError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"livecap status {status}: {msg}")
        self.status = status


def _ptr(a) -> Optional[int]:
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _arr(a, dtype):
    """numpy arrays are converted to a contiguous copy of `dtype`; torch
    tensors must already have the matching dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=dtype)
    return a


class Context:
    """One capture: template, graph, frame and solver state on one GPU."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = load()
        h = _P()
        st = 0
        if stream is not None:
            st = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.lc_create(ctypes.byref(h), device, st), None)
        self.h = h
        self.device = device
        self.N = self.n = self.K = 0
        self.W = self.H = 0
        self.n_dof = 0

    def close(self):
        if getattr(self, "h", None):
            self._lib.lc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st: int, h=0):
        if st != LC_OK:
            msg = "" if h is None else self._lib.lc_last_error(self.h if h == 0 else h).decode()
            raise LivecapError(st, msg)

    # ---- setup
    def params(self) -> lc_params:
        p = lc_params()
        self._lib.lc_params_default(ctypes.byref(p))
        return p

    def set_params(self, **kw):
        p = self.params() if not hasattr(self, "_params") else lc_params.from_buffer_copy(self._params)
        for k, v in kw.items():
            if k == "pyr_ksize":
                v = (ctypes.c_int * 3)(*[int(x) for x in v])
            setattr(p, k, v)
        self._check(self._lib.lc_set_params(self.h, ctypes.byref(p)))
        self._params = p

    def set_camera(self, f, cx, cy, W, H):
        self._check(self._lib.lc_set_camera(self.h, float(f), float(cx), float(cy), int(W), int(H)))
        self.W, self.H = int(W), int(H)

    def upload_template(self, V, tris, albedo, material):
        V = _arr(V, np.float32)
        tris = _arr(tris, np.int32)
        albedo = _arr(albedo, np.float32)
        material = _arr(material, np.float32)
        N, F = len(V), len(tris)
        self._check(self._lib.lc_upload_template(self.h, _ptr(V), N, _ptr(tris), F, _ptr(albedo), _ptr(material)))
        self.N = N

    def build_graph(self, n_nodes: int, K: int):
        self._check(self._lib.lc_build_graph(self.h, int(n_nodes), int(K)))
        self.n, self.K = int(n_nodes), int(K)

    def upload_graph(self, node_vid, bind_idx, bind_w, edge_off, edge_dst, edge_s):
        """A caller-built graph (the layout of read_graph)."""
        node_vid = _arr(node_vid, np.int32)
        bind_idx = _arr(bind_idx, np.int32)
        bind_w = _arr(bind_w, np.float32)
        edge_off = _arr(edge_off, np.int32)
        edge_dst = _arr(edge_dst, np.int32)
        edge_s = _arr(edge_s, np.float32)
        n, K = int(node_vid.shape[0]), int(bind_idx.shape[1])
        self._check(self._lib.lc_upload_graph(self.h, n, K, _ptr(node_vid), _ptr(bind_idx), _ptr(bind_w),
                                              _ptr(edge_off), _ptr(edge_dst), _ptr(edge_s)))
        self.n, self.K = n, K

    def read_graph(self) -> dict:
        ne = ctypes.c_int(0)
        self._check(self._lib.lc_read_graph(self.h, None, None, None, None, None, None, ctypes.byref(ne)))
        E = ne.value
        out = dict(node_vid=np.zeros(self.n, np.int32), bind_idx=np.zeros((self.N, self.K), np.int32),
                   bind_w=np.zeros((self.N, self.K), np.float32), edge_off=np.zeros(self.n + 1, np.int32),
                   edge_dst=np.zeros(E, np.int32), edge_s=np.zeros(E, np.float32))
        self._check(self._lib.lc_read_graph(self.h, *(_ptr(out[k]) for k in
                                                       ("node_vid", "bind_idx", "bind_w", "edge_off",
                                                        "edge_dst", "edge_s")), None))
        return out

    def set_node_params(self, R=None, t=None):
        R = _arr(R, np.float32)
        t = _arr(t, np.float32)
        self._check(self._lib.lc_set_node_params(self.h, _ptr(R), _ptr(t)))

    def set_rest_geometry(self, V_S=None):
        V_S = _arr(V_S, np.float32)
        self._check(self._lib.lc_set_rest_geometry(self.h, _ptr(V_S)))

    def upload_frame(self, rgb, dt, mask, joints2d=None, joints3d=None):
        rgb = _arr(rgb, np.float32)
        dt = _arr(dt, np.float32)
        mask = _arr(mask, np.uint8)
        j2 = _arr(joints2d, np.float32)
        j3 = _arr(joints3d, np.float32)
        self._check(self._lib.lc_upload_frame(self.h, _ptr(rgb), _ptr(dt), _ptr(mask), _ptr(j2), _ptr(j3)))

    def read_frame(self):
        """(dt H x W float32, mask H x W uint8) as the solver samples them."""
        dt = np.zeros((self.H, self.W), np.float32)
        mask = np.zeros((self.H, self.W), np.uint8)
        self._check(self._lib.lc_read_frame(self.h, _ptr(dt), _ptr(mask)))
        return dt, mask

    def set_body_parts(self, bone_part, torso_part: int = 0, dilate_px: int = 10):
        """Body-part mask of the silhouette term (None: off)."""
        bp = _arr(bone_part, np.int32)
        self._check(self._lib.lc_set_body_parts(self.h, _ptr(bp), int(torso_part), int(dilate_px)))

    def read_part_mask(self):
        """(H x W uint8 labels, 255 = none; N uint8 vertex parts)."""
        m = np.zeros((self.H, self.W), np.uint8)
        v = np.zeros(self.N, np.uint8)
        self._check(self._lib.lc_read_part_mask(self.h, _ptr(m), _ptr(v)))
        return m, v

    def read_pyramid_level(self, j: int):
        """Level j (0 coarsest) of the photometric pyramid, (Hj, Wj, 3) float32."""
        Wd, Hd = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._lib.lc_read_pyramid_level(self.h, int(j), None, ctypes.byref(Wd), ctypes.byref(Hd)))
        out = np.zeros((Hd.value, Wd.value, 3), np.float32)
        self._check(self._lib.lc_read_pyramid_level(self.h, int(j), _ptr(out), None, None))
        return out

    # ---- solve
    def solve_nonrigid(self, stats: bool = True):
        if not stats:
            self._check(self._lib.lc_solve_nonrigid(self.h, None))
            return None
        s = lc_solve_stats()
        self._check(self._lib.lc_solve_nonrigid(self.h, ctypes.byref(s)))
        return s.to_dict()

    def read_stats(self) -> dict:
        """Statistics of the last non-rigid solve."""
        st = lc_solve_stats()
        self._check(self._lib.lc_read_stats(self.h, ctypes.byref(st)))
        return st.to_dict()

    def read_back(self, R=True, t=True, V=True, flags=True, pose=False):
        out = {}
        if R:
            out["R"] = np.zeros((self.n, 3, 3), np.float32)
        if t:
            out["t"] = np.zeros((self.n, 3), np.float32)
        if V:
            out["V"] = np.zeros((self.N, 3), np.float32)
        if flags:
            out["flags"] = np.zeros(self.N, np.uint8)
        if pose:
            out["pose"] = np.zeros(self.n_dof, np.float32)
        self._check(self._lib.lc_read_back(self.h, _ptr(out.get("R")), _ptr(out.get("t")), _ptr(out.get("V")),
                                           _ptr(out.get("flags")), _ptr(out.get("pose"))))
        return out

    # ---- learned warm start
    def node_features(self, out=None) -> np.ndarray:
        """Features n x 64 (host array, or ``out``: a device tensor)."""
        F = np.zeros((self.n, 64), np.float32) if out is None else out
        self._check(self._lib.lc_node_features(self.h, _ptr(F)))
        return F

    def record_motion(self):
        self._check(self._lib.lc_record_motion(self.h))

    def read_motion(self, out=None) -> np.ndarray:
        """Motion of the last record_motion, n x 6 (host array, or ``out``:
        a device tensor / pointer-bearing array of n x 6 floats)."""
        u = np.zeros((self.n, 6), np.float32) if out is None else out
        self._check(self._lib.lc_read_motion(self.h, _ptr(u)))
        return u

    def warm_start(self, mlp, sync: bool = True):
        if not sync:
            self._check(self._lib.lc_warm_start(self.h, mlp.h, None, None))
            return None
        acc = ctypes.c_int(0)
        e = np.zeros(2, np.float64)
        self._check(self._lib.lc_warm_start(self.h, mlp.h, ctypes.byref(acc), _ptr(e)))
        return bool(acc.value), e

    # ---- inspection
    def compute_visibility(self):
        self._check(self._lib.lc_compute_visibility(self.h))

    def read_visibility(self) -> dict:
        out = dict(zbuf=np.zeros((self.H, self.W), np.uint64), flags=np.zeros(self.N, np.uint8),
                   uv=np.zeros((self.N, 2), np.float32))
        self._check(self._lib.lc_read_visibility(self.h, _ptr(out["zbuf"]), _ptr(out["flags"]), _ptr(out["uv"])))
        return out

    def eval_linearization(self) -> dict:
        N = self.N
        out = dict(v=np.zeros((N, 3), np.float32), uv=np.zeros((N, 2), np.float32),
                   r_photo=np.zeros((N, 3), np.float32), r_sil=np.zeros(N, np.float32),
                   H=np.zeros((N, 6), np.float32), e=np.zeros((N, 3), np.float32), energy=np.zeros(3))
        self._check(self._lib.lc_eval_linearization(self.h, *(_ptr(out[k]) for k in
                                                               ("v", "uv", "r_photo", "r_sil", "H", "e",
                                                                "energy"))))
        return out

    def eval_gradient(self):
        rhs = np.zeros(6 * self.n, np.float32)
        diag = np.zeros(6 * self.n, np.float32)
        self._check(self._lib.lc_eval_gradient(self.h, _ptr(rhs), _ptr(diag)))
        return rhs, diag

    def apply_jtj(self, p):
        p = _arr(p, np.float32)
        out = np.zeros(6 * self.n, np.float32)
        self._check(self._lib.lc_apply_jtj(self.h, _ptr(p), _ptr(out)))
        return out

    def solve_linear(self):
        d = np.zeros(6 * self.n, np.float32)
        it = ctypes.c_int(0)
        self._check(self._lib.lc_solve_linear(self.h, _ptr(d), ctypes.byref(it)))
        return d, it.value

    # ---- per-vertex surface stage
    def set_surface(self, V):
        V = _arr(V, np.float32)
        self._check(self._lib.lc_set_surface(self.h, _ptr(V)))

    def surface_start(self):
        self._check(self._lib.lc_surface_start(self.h))

    def surface_history(self, V_prev=None, V_prev2=None):
        V_prev = _arr(V_prev, np.float32)
        V_prev2 = _arr(V_prev2, np.float32)
        self._check(self._lib.lc_surface_history(self.h, _ptr(V_prev), _ptr(V_prev2)))

    def surface_advance(self):
        self._check(self._lib.lc_surface_advance(self.h))

    def solve_surface(self, stats: bool = True):
        if not stats:
            self._check(self._lib.lc_solve_surface(self.h, None))
            return None
        s = lc_solve_stats()
        self._check(self._lib.lc_solve_surface(self.h, ctypes.byref(s)))
        return s.to_dict()

    def read_surface(self, flags: bool = False):
        V = np.zeros((self.N, 3), np.float32)
        f = np.zeros(self.N, np.uint8) if flags else None
        self._check(self._lib.lc_read_surface(self.h, _ptr(V), _ptr(f)))
        return (V, f) if flags else V

    def surface_visibility(self):
        self._check(self._lib.lc_surface_visibility(self.h))

    def surface_linearize(self) -> dict:
        out = dict(rhs=np.zeros((self.N, 3), np.float32), diag=np.zeros((self.N, 3), np.float32),
                   energy=np.zeros(6))
        self._check(self._lib.lc_surface_linearize(self.h, _ptr(out["rhs"]), _ptr(out["diag"]),
                                                   _ptr(out["energy"])))
        return out

    def surface_apply_jtj(self, p):
        p = _arr(p, np.float32)
        out = np.zeros((self.N, 3), np.float32)
        self._check(self._lib.lc_surface_apply_jtj(self.h, _ptr(p), _ptr(out)))
        return out

    def surface_solve_linear(self):
        d = np.zeros((self.N, 3), np.float32)
        it = ctypes.c_int(0)
        self._check(self._lib.lc_surface_solve_linear(self.h, _ptr(d), ctypes.byref(it)))
        return d, it.value

    # ---- profiling
    def set_profiling(self, on: bool):
        self._check(self._lib.lc_set_profiling(self.h, 1 if on else 0))

    def read_profile(self) -> dict:
        ms = np.zeros(len(PHASES), np.float64)
        cnt = np.zeros(len(PHASES), np.int32)
        self._check(self._lib.lc_read_profile(self.h, _ptr(ms), _ptr(cnt)))
        return {name: (float(ms[j]), int(cnt[j])) for j, name in enumerate(PHASES)}

    # ---- pose stage
    def upload_skeleton(self, parents, joints_rest, dof, skin_idx, skin_w):
        parents = _arr(parents, np.int32)
        joints_rest = _arr(joints_rest, np.float32)
        dof = _arr(dof, np.uint8)
        skin_idx = _arr(skin_idx, np.int32)
        skin_w = _arr(skin_w, np.float32)
        J = len(parents)
        self._check(self._lib.lc_upload_skeleton(self.h, J, _ptr(parents), _ptr(joints_rest), _ptr(dof),
                                                 _ptr(skin_idx), _ptr(skin_w)))
        self.n_dof = 6 + 3 * int(np.count_nonzero(np.asarray(dof)[1:]))

    def set_pose(self, pose):
        pose = _arr(pose, np.float32)
        self._check(self._lib.lc_set_pose(self.h, _ptr(pose)))

    def reset_pose(self):
        """Restart from the pose last given to set_pose (device-side, no sync)."""
        self._check(self._lib.lc_reset_pose(self.h))

    def set_pose_priors(self, temporal_w=None, theta_min=None, theta_max=None):
        w = _arr(temporal_w, np.float32)
        lo = _arr(theta_min, np.float32)
        hi = _arr(theta_max, np.float32)
        self._check(self._lib.lc_set_pose_priors(self.h, _ptr(w), _ptr(lo), _ptr(hi)))

    def pose_advance(self):
        self._check(self._lib.lc_pose_advance(self.h))

    def pose_extrapolate(self):
        self._check(self._lib.lc_pose_extrapolate(self.h))

    def pose_clear_history(self):
        self._check(self._lib.lc_pose_clear_history(self.h))

    def eval_pose(self) -> dict:
        nd = self.n_dof
        out = dict(V=np.zeros((self.N, 3), np.float32), A=np.zeros((nd, nd)), g=np.zeros(nd), energy=np.zeros(1))
        self._check(self._lib.lc_eval_pose(self.h, _ptr(out["V"]), _ptr(out["A"]), _ptr(out["g"]),
                                           _ptr(out["energy"])))
        return out

    def solve_pose(self, stats: bool = True):
        if not stats:
            self._check(self._lib.lc_solve_pose(self.h, None))
            return None
        s = lc_solve_stats()
        self._check(self._lib.lc_solve_pose(self.h, ctypes.byref(s)))
        return s.to_dict()


MLP_PARAMS = 83974


class MLP:
    """The warm-start network (lc_mlp_*): 64 -> 256 -> 256 -> 6, BF16 tensor-core
    kernels, FP32 master parameters, Adam."""

    def __init__(self, device: int = 0, params=None, mu=None, sigma=None):
        self._lib = load()
        self.device = device
        self._keep = [_arr(params, np.float32), _arr(mu, np.float32), _arr(sigma, np.float32)]
        h = _P()
        st = self._lib.lc_mlp_create(ctypes.byref(h), device, *[_ptr(a) for a in self._keep])
        if st != LC_OK:
            raise LivecapError(st, "lc_mlp_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.lc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != LC_OK:
            raise LivecapError(st, self._lib.lc_mlp_last_error(self.h).decode())

    def params(self) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, np.float32)
        self._check(self._lib.lc_mlp_get_params(self.h, _ptr(out)))
        return out

    def set_gemm(self, kind: int):
        """GEMM_TCGEN05 (default) or GEMM_MMA_SYNC."""
        self._check(self._lib.lc_mlp_set_gemm(self.h, int(kind)))

    def set_scaling(self, mu=None, sigma=None, s_out=None):
        keep = [_arr(a, np.float32) for a in (mu, sigma, s_out)]
        self._check(self._lib.lc_mlp_set_scaling(self.h, *[_ptr(a) for a in keep]))

    def scaling(self):
        """(mu, sigma, s_out) as host arrays."""
        mu, sigma, s_out = np.zeros(64, np.float32), np.zeros(64, np.float32), np.zeros(6, np.float32)
        self._check(self._lib.lc_mlp_get_scaling(self.h, _ptr(mu), _ptr(sigma), _ptr(s_out)))
        return mu, sigma, s_out

    def fit_scaling(self, F_dev, T_dev):
        """mu / sigma / s_out from device arrays F (rows x 64), T (rows x 6)."""
        self._check(self._lib.lc_mlp_fit_scaling(self.h, _ptr(F_dev), _ptr(T_dev), int(F_dev.shape[0])))

    def forward(self, F) -> np.ndarray:
        F = _arr(F, np.float32)
        Y = np.zeros((F.shape[0], 6), np.float32)
        self._check(self._lib.lc_mlp_forward(self.h, _ptr(F), F.shape[0], _ptr(Y)))
        return Y

    def gradient(self, F, T):
        F, T = _arr(F, np.float32), _arr(T, np.float32)
        g = np.zeros(MLP_PARAMS, np.float32)
        loss = ctypes.c_double(0.0)
        self._check(self._lib.lc_mlp_gradient(self.h, _ptr(F), _ptr(T), F.shape[0], _ptr(g), ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, F_dev, T_dev, idx, lr: float, want_loss: bool = False):
        """One Adam step on rows idx of device arrays F_dev (rows x 64), T_dev (rows x 6)."""
        idx = _arr(idx, np.int32)
        loss = ctypes.c_double(0.0)
        self._check(self._lib.lc_mlp_train_step(self.h, _ptr(F_dev), _ptr(T_dev), _ptr(idx), len(idx),
                                                float(lr), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


STEP_EULER_START, STEP_CARRY_GRAPH = 1, 2
GEMM_TCGEN05, GEMM_MMA_SYNC = 0, 1
BATCH_PCG_AUTO, BATCH_PCG_CLUSTER8, BATCH_PCG_CLUSTER16, BATCH_PCG_PER_ITERATION = 0, 1, 2, 3


class lc_batch_shape(ctypes.Structure):
    _fields_ = [("pcg_mode", ctypes.c_int), ("vert_block", ctypes.c_int), ("node_warps", ctypes.c_int),
                ("node_unroll", ctypes.c_int)]

    def to_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def autotune_table() -> str:
    """The process-wide shape table (lc_autotune_table) as text."""
    lib = load()
    need = ctypes.c_int(0)
    if lib.lc_autotune_table(None, 0, ctypes.byref(need)) != LC_OK:
        raise LivecapError(LC_ERR_ARG, "lc_autotune_table failed")
    buf = ctypes.create_string_buffer(max(need.value, 1))
    if lib.lc_autotune_table(buf, len(buf), None) != LC_OK:
        raise LivecapError(LC_ERR_ARG, "lc_autotune_table failed")
    return buf.value.decode()


def autotune_table_load(text: str):
    st = load().lc_autotune_table_load(text.encode())
    if st != LC_OK:
        raise LivecapError(st, "lc_autotune_table_load: malformed table")


class Batch:
    """Several contexts solved together (lc_batch_*): one launch per phase
    for all captures, the whole non-rigid loop in one CUDA graph."""

    def __init__(self, contexts):
        self._lib = load()
        self.contexts = list(contexts)
        arr = (_P * len(self.contexts))(*[c.h for c in self.contexts])
        h = _P()
        st = self._lib.lc_batch_create(ctypes.byref(h), arr, len(self.contexts))
        if st != LC_OK:
            raise LivecapError(st, self._lib.lc_last_error(self.contexts[0].h).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.lc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != LC_OK:
            raise LivecapError(st, self._lib.lc_batch_last_error(self.h).decode())

    def set_pcg_mode(self, mode: int):
        self._check(self._lib.lc_batch_set_pcg_mode(self.h, int(mode)))

    def solve(self, from_identity: bool = True, stats: bool = True):
        if not stats:
            self._check(self._lib.lc_batch_solve(self.h, int(from_identity), None))
            return None
        arr = (lc_solve_stats * len(self.contexts))()
        self._check(self._lib.lc_batch_solve(self.h, int(from_identity), arr))
        return [a.to_dict() for a in arr]

    @property
    def stream_handle(self) -> int:
        """The batch's cudaStream_t as an integer."""
        return self._lib.lc_batch_stream(self.h) or 0

    def step(self, mlp=None, euler_start: bool = True, carry_graph: bool = True, stats: bool = True):
        """One frame step of every member as one CUDA graph (lc_batch_step):
        pose stage, identity start of the non-rigid stage unless
        ``carry_graph``, warm start (with ``mlp``), batched non-rigid stage,
        motion and pose bookkeeping.  Returns per-member non-rigid statistics."""
        flags = (STEP_EULER_START if euler_start else 0) | (STEP_CARRY_GRAPH if carry_graph else 0)
        h = mlp.h if mlp is not None else None
        if not stats:
            self._check(self._lib.lc_batch_step(self.h, h, flags, None))
            return None
        arr = (lc_solve_stats * len(self.contexts))()
        self._check(self._lib.lc_batch_step(self.h, h, flags, arr))
        return [a.to_dict() for a in arr]

    def set_shape(self, pcg_mode: int, vert_block: int = 256, node_warps: int = 4, node_unroll: int = 4):
        sh = lc_batch_shape(pcg_mode, vert_block, node_warps, node_unroll)
        self._check(self._lib.lc_batch_set_shape(self.h, ctypes.byref(sh)))

    def shape(self) -> dict:
        sh = lc_batch_shape()
        self._check(self._lib.lc_batch_get_shape(self.h, ctypes.byref(sh)))
        return sh.to_dict()

    def size_class(self) -> str:
        buf = ctypes.create_string_buffer(4096)
        self._check(self._lib.lc_batch_size_class(self.h, buf, len(buf)))
        return buf.value.decode()

    def autotune_shapes(self, reps: int = 2, use_cache: bool = True) -> dict:
        """lc_batch_autotune_shapes: returns the chosen shape, its time and
        whether it came from the table, with the counts of shapes tried and
        rejected by the bit-identity check."""
        sh = lc_batch_shape()
        ms = ctypes.c_float(0.0)
        hit, tried, rej = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._lib.lc_batch_autotune_shapes(self.h, int(reps), int(use_cache), ctypes.byref(sh),
                                                       ctypes.byref(ms), ctypes.byref(hit), ctypes.byref(tried),
                                                       ctypes.byref(rej)))
        return dict(shape=sh.to_dict(), ms=ms.value, from_cache=bool(hit.value), tried=tried.value,
                    rejected=rej.value)

    def apply_jtj(self, stage: bool = False):
        """Enqueue one J^T J p of every member (measurement entry); stage
        recomputes the operands it reads first."""
        self._check(self._lib.lc_batch_apply_jtj(self.h, int(stage)))

    def autotune(self, reps: int = 3):
        mode = ctypes.c_int(-1)
        ms = np.zeros(4, np.float32)
        self._check(self._lib.lc_batch_autotune(self.h, int(reps), ctypes.byref(mode), _ptr(ms)))
        return mode.value, ms
