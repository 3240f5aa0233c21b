"""Non-rigid stage in FP64: warp, residuals, Jacobian, PCG, Gauss-Newton.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What it computes (paper references are to sections and equations):

* Energy (Sec. 3.4, E_non-rigid = E_data + E_reg, data terms E_photo and
  E_silhouette) with the embedded-graph regulariser the solver targets:

      E = w_p sum_{i in V} ||I(pi(v'_i)) - C_i||^2
        + w_s sum_{i in B} I_DT(pi(v'_i))^2
        + w_a sum_{(k,l)} s_kl ||R_k (g_l - g_k) + g_k + t_k - (g_l + t_l)||^2

  with the warp v'_i = v_i + sum_s w_is ((R_k - I)(v_i - g_k) + t_k), k = the
  s-th node bound to vertex i (the normalised-weight form of
  sum_s w_is (R_k (v_i - g_k) + g_k + t_k)), and the pinhole projection
  pi(X,Y,Z) = (f X/Z + cx, f Y/Z + cy) (Sec. 3.3, full perspective camera).
* The robust colour kernel sigma_c (Sec. 3.4) is off by default (its
  threshold is not given); when on, it zeroes the photometric rows of a
  correspondence whose colour differs by more than sigma_c.  The
  photometric term samples the raw image by default, or the Gaussian
  pyramid of module ``pyramid`` with one Gauss-Newton iteration per level.
  With a body-part mask (module ``parts``) a contour vertex whose projection
  lands on another part's region has no silhouette residual there.
* Sampling: bilinear, clamp to edge, lerp(a,b,t) = a + t (b - a); image
  gradients are central differences (one-sided at the border) sampled
  bilinearly.  Vertices with Z <= 1e-3 or a projection outside
  [0,W-1] x [0,H-1] contribute no residual at that linearisation.
* Visibility V and the contour set B are fixed per frame (Sec. 3.3 and 3.4);
  the direction b_i of each contour vertex is re-evaluated at every
  linearisation from the current surface (its normal and the DT gradient at
  its projection), so that a vertex which crossed the medial axis follows the
  contour it now faces.  Both come from the exact-arithmetic module
  ``visibility``.
* The silhouette residual is r_i = sqrt(w_s) I_DT(pi(v'_i)); its Jacobian row
  is multiplied by b_i, so b_i = -1 reverses the row's pull along the DT
  gradient (Sec. 3.3, the two silhouette cases) while J^T J stays PSD.
  b_i = -1 only for contour vertices that project inside the foreground and
  whose projected normal opposes z = -grad(I_DT).
* Unknowns per node: (d_omega, d_t); rotations update on the left,
  R_k <- Exp(d_omega) R_k, translations add.  Gauss-Newton without damping
  or line search (Sec. 4, Eq. normal equations; no residual evaluation
  inside the iterations), the linear system solved by Jacobi-preconditioned
  CG from x0 = 0 for a fixed number of iterations (Sec. 4, non-rigid
  registration).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp

from . import parts as _parts
from . import pyramid as _pyr


# ----------------------------------------------------------------------------
# SO(3)
# ----------------------------------------------------------------------------
def hat(a: np.ndarray) -> np.ndarray:
    """Skew matrices [a]_x with [a]_x b = a x b; a (...,3) -> (...,3,3)."""
    a = np.asarray(a, dtype=np.float64)
    z = np.zeros(a.shape[:-1])
    return np.stack([
        np.stack([z, -a[..., 2], a[..., 1]], -1),
        np.stack([a[..., 2], z, -a[..., 0]], -1),
        np.stack([-a[..., 1], a[..., 0], z], -1)], -2)


def so3_exp(w: np.ndarray) -> np.ndarray:
    """Rodrigues' formula, (n,3) -> (n,3,3)."""
    w = np.atleast_2d(np.asarray(w, dtype=np.float64))
    th = np.linalg.norm(w, axis=1)
    W = hat(w)
    W2 = W @ W
    small = th < 1e-8
    ths = np.where(small, 1.0, th)
    A = np.where(small, 1.0 - th * th / 6.0, np.sin(ths) / ths)
    B = np.where(small, 0.5 - th * th / 24.0, (1.0 - np.cos(ths)) / (ths * ths))
    return np.eye(3)[None] + A[:, None, None] * W + B[:, None, None] * W2


def so3_log(R: np.ndarray) -> np.ndarray:
    """Axis-angle of rotations (n,3,3) -> (n,3), angle in [0, pi] (SciPy)."""
    from scipy.spatial.transform import Rotation
    return Rotation.from_matrix(np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)).as_rotvec()


# ----------------------------------------------------------------------------
# Problem data
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """One capture's frame-fixed data, all promoted to FP64."""

    base: np.ndarray        # (N,3) rest geometry of this stage
    albedo: np.ndarray      # (N,3)
    g: np.ndarray           # (n,3) node positions (base[node_vid])
    bind_idx: np.ndarray    # (N,K)
    bind_w: np.ndarray      # (N,K)
    edges: np.ndarray       # (E,2) directed
    edge_s: np.ndarray      # (E,)
    f: float
    cx: float
    cy: float
    W: int
    H: int
    rgb: np.ndarray         # (H,W,3)
    dt: np.ndarray          # (H,W)
    mask: np.ndarray        # (H,W) foreground silhouette
    w_photo: float
    w_sil: float
    w_arap: float
    vis: Optional[np.ndarray] = None     # (N,) bool
    inB: Optional[np.ndarray] = None     # (N,) bool
    bsign: Optional[np.ndarray] = None   # (N,) +-1
    tris: Optional[np.ndarray] = None    # (T,3): when set, b_i follows the current surface
    sigma_c: float = 0.0                 # robust colour kernel threshold (0: off)
    pruned: Optional[np.ndarray] = None  # (N,) given pruning decisions (None: decide here)
    pyr_levels: int = 0                  # photometric pyramid levels (0: raw image)
    pyr_ksize: tuple = _pyr.DEFAULT_KSIZE
    level: Optional[int] = None          # pyramid level sampled now (None: raw image)
    part_mask: Optional[np.ndarray] = None   # (H,W) uint8 body-part mask of V^S (None: off)
    vpart: Optional[np.ndarray] = None       # (N,) uint8 part of every vertex

    @property
    def n(self) -> int:
        return len(self.g)

    def __post_init__(self):
        f64 = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
        self.base, self.albedo, self.g = f64(self.base), f64(self.albedo), f64(self.g)
        self.bind_w, self.edge_s = f64(self.bind_w), f64(self.edge_s)
        self.rgb, self.dt = f64(self.rgb), f64(self.dt)
        self.bind_idx = np.asarray(self.bind_idx, dtype=np.int64)
        self.edges = np.asarray(self.edges, dtype=np.int64).reshape(-1, 2)
        self._grad_rgb = None
        self._grad_dt = None

    def grads(self):
        if self._grad_rgb is None:
            self._grad_rgb = central_differences(self.rgb)
            self._grad_dt = central_differences(self.dt)
        return self._grad_rgb, self._grad_dt


def identity_params(n: int):
    return np.tile(np.eye(3), (n, 1, 1)), np.zeros((n, 3))


# ----------------------------------------------------------------------------
# Warp, projection, sampling
# ----------------------------------------------------------------------------
def warp(P: Problem, R: np.ndarray, t: np.ndarray) -> np.ndarray:
    """v'_i = v_i + sum_s w_is ((R_k - I)(v_i - g_k) + t_k)."""
    v = P.base
    out = v.copy()
    I3 = np.eye(3)
    for s in range(P.bind_idx.shape[1]):
        k = P.bind_idx[:, s]
        rel = v - P.g[k]
        disp = np.einsum("nij,nj->ni", R[k] - I3, rel) + t[k]
        out += P.bind_w[:, s, None] * disp
    return out


def project(P: Problem, v: np.ndarray):
    """(u, v) pixel coordinates, validity (Z > 1e-3) and in-image flag."""
    X, Y, Z = v[:, 0], v[:, 1], v[:, 2]
    valid = Z > 1e-3
    Zs = np.where(valid, Z, 1.0)
    u = P.f * X / Zs + P.cx
    w = P.f * Y / Zs + P.cy
    inimg = valid & (u >= 0) & (u <= P.W - 1) & (w >= 0) & (w <= P.H - 1)
    return u, w, valid, inimg


def central_differences(img: np.ndarray):
    """(d/dx, d/dy): (I[x+1]-I[x-1])/2 inside, one-sided at the border."""
    img = np.asarray(img, dtype=np.float64)
    gx = np.zeros_like(img)
    gy = np.zeros_like(img)
    if img.shape[1] >= 2:
        gx[:, 1:-1] = (img[:, 2:] - img[:, :-2]) * 0.5
        gx[:, 0] = img[:, 1] - img[:, 0]
        gx[:, -1] = img[:, -1] - img[:, -2]
    if img.shape[0] >= 2:
        gy[1:-1] = (img[2:] - img[:-2]) * 0.5
        gy[0] = img[1] - img[0]
        gy[-1] = img[-1] - img[-2]
    return gx, gy


def photo_level(P, j: int):
    """Level j of the photometric pyramid and its central differences,
    cached for the problem's current image."""
    key = (tuple(int(k) for k in P.pyr_ksize), j)
    cache = P.__dict__.get("_pyr_cache")
    if cache is None or cache[0] is not P.rgb:
        cache = (P.rgb, {})
        P._pyr_cache = cache
    if key not in cache[1]:
        img = _pyr.level_image(P.rgb, j, P.pyr_ksize)
        cache[1][key] = (img, central_differences(img))
    return cache[1][key]


def photo_sample(P, u: np.ndarray, v: np.ndarray, grad: bool = False):
    """Colour I(u, v) (m,3) sampled for the photometric term at full-resolution
    coordinates, from the raw image or the current pyramid level; with grad,
    also d I / d(u, v) (m,3,2) in full-resolution pixels."""
    j = getattr(P, "level", None)
    if j is None:
        I = bilinear(P.rgb, u, v)
        if not grad:
            return I
        gx, gy = P.grads()[0]
        return I, np.stack([bilinear(gx, u, v), bilinear(gy, u, v)], axis=2)
    img, (gx, gy) = photo_level(P, j)
    uj, vj = _pyr.to_level(u, j), _pyr.to_level(v, j)
    I = bilinear(img, uj, vj)
    if not grad:
        return I
    d = float(_pyr.FACTORS[j])
    return I, np.stack([bilinear(gx, uj, vj), bilinear(gy, uj, vj)], axis=2) / d


def bilinear(img: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Bilinear sample with clamp to edge; lerp(a,b,t) = a + t(b-a)."""
    H, W = img.shape[:2]
    uc = np.clip(u, 0.0, W - 1)
    vc = np.clip(v, 0.0, H - 1)
    x0 = np.floor(uc).astype(np.int64)
    y0 = np.floor(vc).astype(np.int64)
    fx = uc - x0
    fy = vc - y0
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    if img.ndim == 3:
        fx = fx[:, None]
        fy = fy[:, None]
    a, b = img[y0, x0], img[y0, x1]
    c, d = img[y1, x0], img[y1, x1]
    top = a + fx * (b - a)
    bot = c + fx * (d - c)
    return top + fy * (bot - top)


def dproj(P: Problem, v: np.ndarray) -> np.ndarray:
    """d pi / d v' (N,2,3)."""
    X, Y, Z = v[:, 0], v[:, 1], v[:, 2]
    Zs = np.where(Z > 1e-3, Z, 1.0)
    out = np.zeros((len(v), 2, 3))
    out[:, 0, 0] = P.f / Zs
    out[:, 0, 2] = -P.f * X / (Zs * Zs)
    out[:, 1, 1] = P.f / Zs
    out[:, 1, 2] = -P.f * Y / (Zs * Zs)
    return out


# ----------------------------------------------------------------------------
# Residuals and Jacobian
# ----------------------------------------------------------------------------
def prune(P, photo_on: np.ndarray, u: np.ndarray, w: np.ndarray) -> np.ndarray:
    """The robust colour kernel sigma_c (Sec. 3.4): photometric
    correspondences whose colour difference ||I(pi(v)) - C|| exceeds sigma_c
    are dropped (their residual and Jacobian rows are zero).  P.pruned, when
    given, holds the decisions instead (taken in FP32 by the kernel; the
    FP64 distance here differs from it only within rounding of sigma_c)."""
    if not getattr(P, "sigma_c", 0.0) > 0.0:
        return photo_on
    if P.pruned is not None:
        return photo_on & ~np.asarray(P.pruned, dtype=bool)
    out = photo_on.copy()
    idx = np.nonzero(photo_on)[0]
    if len(idx):
        d = np.linalg.norm(photo_sample(P, u[idx], w[idx]) - P.albedo[idx], axis=1)
        out[idx] = d <= P.sigma_c
    return out



def vertex_residuals(P: Problem, R: np.ndarray, t: np.ndarray) -> dict:
    """Per-vertex data residuals at the given parameters.

    photo (N,3) = sqrt(w_p)(I(uv) - C) where photometrically active, else 0;
    sil (N,)    = sqrt(w_s) DT(uv) where in B and active, else 0.
    """
    v = warp(P, R, t)
    u, w, valid, inimg = project(P, v)
    photo_on = prune(P, inimg & P.vis, u, w)
    sil_on = inimg & P.inB & ~_parts.masked(P, v)
    photo = np.zeros((len(v), 3))
    sil = np.zeros(len(v))
    if photo_on.any():
        photo[photo_on] = np.sqrt(P.w_photo) * (photo_sample(P, u[photo_on], w[photo_on])
                                                - P.albedo[photo_on])
    if sil_on.any():
        sil[sil_on] = np.sqrt(P.w_sil) * bilinear(P.dt, u[sil_on], w[sil_on])
    return dict(v=v, u=u, w=w, photo=photo, sil=sil, photo_on=photo_on, sil_on=sil_on)


def arap_residuals(P: Problem, R: np.ndarray, t: np.ndarray) -> np.ndarray:
    """(E,3) residuals sqrt(w_a s_kl)(R_k(g_l-g_k) + g_k + t_k - g_l - t_l)."""
    k, l = P.edges[:, 0], P.edges[:, 1]
    b = np.einsum("eij,ej->ei", R[k], P.g[l] - P.g[k])
    d = b + P.g[k] + t[k] - P.g[l] - t[l]
    return np.sqrt(P.w_arap * P.edge_s)[:, None] * d


def energy(P: Problem, R: np.ndarray, t: np.ndarray) -> dict:
    vr = vertex_residuals(P, R, t)
    ar = arap_residuals(P, R, t)
    e = dict(photo=float((vr["photo"] ** 2).sum()), sil=float((vr["sil"] ** 2).sum()),
             arap=float((ar ** 2).sum()))
    e["total"] = e["photo"] + e["sil"] + e["arap"]
    return e


def update_directions(P: Problem, R: np.ndarray, t: np.ndarray):
    """b_i of the frame's contour set at the current FP32 surface."""
    if P.tris is None or P.inB is None:
        return
    from . import visibility as _vis
    v32 = warp(P, R, t).astype(np.float32)
    neg = _vis.directions(v32, P.tris, P.f, P.cx, P.cy, P.W, P.H, P.dt.astype(np.float32), P.mask, P.inB)
    P.bsign = np.where(neg, -1.0, 1.0)


def linearise(P: Problem, R: np.ndarray, t: np.ndarray):
    """Stacked residual vector F and its Jacobian J (sparse, FP64).

    Column 6k..6k+2 is node k's rotation increment, 6k+3..6k+5 its
    translation increment.  Rows: photometric (3 per active vertex, vertex
    order), silhouette (1 per active contour vertex), ARAP (3 per edge).
    """
    n = P.n
    K = P.bind_idx.shape[1]
    update_directions(P, R, t)
    vr = vertex_residuals(P, R, t)
    v, u, w = vr["v"], vr["u"], vr["w"]
    gxD, gyD = P.grads()[1]
    Dp = dproj(P, v)
    rows, cols, vals, Fs = [], [], [], []
    row0 = 0

    def node_blocks(ids, A):
        # A: (m, rdim, 3) = d r / d v'_i; returns COO pieces for all K slots
        m, rdim = A.shape[0], A.shape[1]
        for s in range(K):
            k = P.bind_idx[ids, s]
            a = np.einsum("nij,nj->ni", R[k], P.base[ids] - P.g[k])
            dv = np.concatenate([-hat(a), np.broadcast_to(np.eye(3), (m, 3, 3))], axis=2)
            blk = P.bind_w[ids, s, None, None] * (A @ dv)           # (m, rdim, 6)
            rr = row0 + np.arange(m)[:, None, None] * rdim + np.arange(rdim)[None, :, None]
            cc = 6 * k[:, None, None] + np.arange(6)[None, None, :]
            rows.append(np.broadcast_to(rr, blk.shape).ravel())
            cols.append(np.broadcast_to(cc, blk.shape).ravel())
            vals.append(blk.ravel())

    ip = np.nonzero(vr["photo_on"])[0]
    if len(ip):
        G = photo_sample(P, u[ip], w[ip], grad=True)[1]                     # (m,3,2)
        A = np.sqrt(P.w_photo) * (G @ Dp[ip])
        node_blocks(ip, A)
        Fs.append(vr["photo"][ip].ravel())
        row0 += 3 * len(ip)
    isl = np.nonzero(vr["sil_on"])[0]
    if len(isl):
        G = np.stack([bilinear(gxD, u[isl], w[isl]), bilinear(gyD, u[isl], w[isl])], axis=1)[:, None, :]
        A = (np.sqrt(P.w_sil) * P.bsign[isl])[:, None, None] * (G @ Dp[isl])
        node_blocks(isl, A)
        Fs.append(vr["sil"][isl])
        row0 += len(isl)
    E = len(P.edges)
    if E:
        k, l = P.edges[:, 0], P.edges[:, 1]
        sc = np.sqrt(P.w_arap * P.edge_s)
        b = np.einsum("eij,ej->ei", R[k], P.g[l] - P.g[k])
        blk_w = -sc[:, None, None] * hat(b)
        blk_tk = sc[:, None, None] * np.eye(3)[None]
        rr = row0 + 3 * np.arange(E)[:, None, None] + np.arange(3)[None, :, None]
        for blk, c0 in ((blk_w, 6 * k), (blk_tk, 6 * k + 3), (-blk_tk, 6 * l + 3)):
            cc = c0[:, None, None] + np.arange(3)[None, None, :]
            rows.append(np.broadcast_to(rr, blk.shape).ravel())
            cols.append(np.broadcast_to(cc, blk.shape).ravel())
            vals.append(blk.ravel())
        Fs.append(arap_residuals(P, R, t).ravel())
        row0 += 3 * E
    Fv = np.concatenate(Fs) if Fs else np.zeros(0)
    if rows:
        J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(row0, 6 * n)).tocsr()
    else:
        J = sp.csr_matrix((0, 6 * n))
    return Fv, J


# ----------------------------------------------------------------------------
# Linear solve and Gauss-Newton
# ----------------------------------------------------------------------------
def pcg(A, b: np.ndarray, n_iter: int):
    """Jacobi-preconditioned CG from x0 = 0 for exactly n_iter iterations.

    M^-1 = 1/diag(A) where diag(A) > 0, else 0.  Stops early (flag
    ``breakdown``) if p^T A p <= 0, and stops when r^T z becomes 0.
    """
    d = np.asarray(A.diagonal(), dtype=np.float64)
    minv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    x = np.zeros_like(b)
    r = b.copy()
    z = minv * r
    p = z.copy()
    rz = float(r @ z)
    info = dict(iters=0, breakdown=False, rz=[rz])
    if rz == 0.0:
        return x, info
    for it in range(n_iter):
        Ap = A @ p
        pAp = float(p @ Ap)
        if not pAp > 0.0:
            info["breakdown"] = True
            break
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        z = minv * r
        rz_new = float(r @ z)
        info["iters"] = it + 1
        info["rz"].append(rz_new)
        if rz_new == 0.0:
            break
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, info


def normal_equations(P: Problem, R: np.ndarray, t: np.ndarray):
    """(J^T J, -J^T F, F, J) at the given parameters."""
    F, J = linearise(P, R, t)
    JT = J.T.tocsr()
    return (JT @ J).tocsr(), -(JT @ F), F, J


def apply_update(R: np.ndarray, t: np.ndarray, delta: np.ndarray):
    d = delta.reshape(-1, 6)
    return so3_exp(d[:, :3]) @ R, t + d[:, 3:]


def gauss_newton(P: Problem, R: np.ndarray, t: np.ndarray, n_gn: int, n_pcg: int):
    """Fixed-count Gauss-Newton (no damping, no line search)."""
    hist = []
    for gn in range(n_gn):
        P.level = _pyr.level_of(gn, P.pyr_levels)
        A, b, F, _ = normal_equations(P, R, t)
        delta, info = pcg(A, b, n_pcg)
        hist.append(dict(energy=float(F @ F), step_norm=float(np.linalg.norm(delta)),
                         pcg_iters=info["iters"], breakdown=info["breakdown"]))
        R, t = apply_update(R, t, delta)
    P.level = final_level(P)
    return R, t, hist


def final_level(P):
    """Level of the energy after the last update: the finest one."""
    return _pyr.level_of(1 << 20, P.pyr_levels)


# ----------------------------------------------------------------------------
# Assembling a problem from scene data
# ----------------------------------------------------------------------------
def frame_decisions(P: Problem, tris: np.ndarray, R: np.ndarray, t: np.ndarray, eps=1e-2):
    """Visibility, B and b_i at the given parameters: the FP64 warp rounded
    to FP32, then the exact-arithmetic module."""
    from . import visibility as _vis
    v32 = warp(P, R, t).astype(np.float32)
    out = _vis.visibility(v32, tris, P.f, P.cx, P.cy, P.W, P.H, P.dt.astype(np.float32),
                          P.mask, eps)
    fl = out["flags"]
    P.vis = (fl & _vis.FLAG_VISIBLE) != 0
    P.inB = (fl & _vis.FLAG_INB) != 0
    P.bsign = np.where((fl & _vis.FLAG_BNEG) != 0, -1.0, 1.0)
    return out


def problem_from_scene(scene, graph: dict, base32: Optional[np.ndarray] = None) -> Problem:
    """Problem for a scene (``synth.Scene``) and a graph from ``oracle.graph``.

    ``base32`` is the stage's rest geometry (the template, or the skinned mesh
    after the pose stage); node positions are base[node_vid]."""
    base = np.asarray(scene.V if base32 is None else base32, dtype=np.float32)
    wp, ws, wa = scene.weights
    return Problem(
        base=base.astype(np.float64), albedo=scene.albedo,
        g=base[graph["node_vid"]].astype(np.float64),
        bind_idx=graph["bind_idx"], bind_w=np.asarray(graph["bind_w"], dtype=np.float32),
        edges=graph["edges"], edge_s=np.asarray(graph["edge_s"], dtype=np.float32),
        f=float(np.float32(scene.cam.f)), cx=float(np.float32(scene.cam.cx)),
        cy=float(np.float32(scene.cam.cy)), W=scene.cam.W, H=scene.cam.H,
        rgb=scene.rgb, dt=scene.dt, mask=scene.mask, tris=np.asarray(scene.F, dtype=np.int32), w_photo=wp, w_sil=ws, w_arap=wa)


def solve_scene(scene, graph: Optional[dict] = None, base32=None, n_gn=None, n_pcg=None,
                sigma_c: float = 0.0, pyr_levels: int = 0, pyr_ksize=_pyr.DEFAULT_KSIZE,
                part_mask=None, vpart=None):
    """Whole non-rigid solve from identity parameters (``sigma_c``: the robust
    colour kernel's threshold, 0 = off; ``pyr_levels``: photometric pyramid
    levels, 0 = raw image; ``part_mask`` / ``vpart``: the body-part mask of
    the silhouette term, None = off).  Returns a dict."""
    from . import graph as _graph
    if graph is None:
        graph = _graph.build_graph(scene.V, scene.material, scene.n_nodes, scene.K)
    P = problem_from_scene(scene, graph, base32)
    P.sigma_c = float(sigma_c)
    P.pyr_levels, P.pyr_ksize = int(pyr_levels), tuple(pyr_ksize)
    P.part_mask, P.vpart = part_mask, vpart
    R, t = identity_params(P.n)
    frame_decisions(P, scene.F, R, t)
    P.level = _pyr.level_of(0, P.pyr_levels)
    e0 = energy(P, R, t)
    R, t, hist = gauss_newton(P, R, t, scene.n_gn if n_gn is None else n_gn,
                              scene.n_pcg if n_pcg is None else n_pcg)
    e1 = energy(P, R, t)
    return dict(problem=P, graph=graph, R=R, t=t, hist=hist, e0=e0, e1=e1, v=warp(P, R, t))
