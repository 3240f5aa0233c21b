"""Per-vertex non-rigid surface registration in FP64 (the paper's own
unknowns: the vertex positions V).

TEST INFRASTRUCTURE ONLY (see the package docstring).

What it computes (Sec. 3.4, E_non-rigid = E_data + E_reg with
E_reg = E_smooth + E_edge + E_velocity + E_acceleration; Sec. 4, Gauss-Newton
on the normal equations with a Jacobi-preconditioned CG of fixed length):

    E(V) = w_p  sum_{i in V} ||I(pi(V_i)) - C_i||^2
         + w_s  sum_{i in B} I_DT(pi(V_i))^2                 (row scaled by b_i)
         + w_sm sum_i sum_{j in N_i} s_ij/|N_i| ||(V_i - V_j) - (V^S_i - V^S_j)||^2
         + w_ed sum_i sum_{j in N_i} s_ij/|N_i| (||V_i - V_j|| - ||Vh_i - Vh_j||)^2
         + w_v  sum_i ||V_i - V^{t-1}_i||^2
         + w_a  sum_i ||V_i - 2 V^{t-1}_i + V^{t-2}_i||^2

Readings of points the paper leaves open:

* N_i is the one-ring of vertex i (the vertices that share a mesh edge with
  it); every ordered pair (i, j in N_i) is one residual of E_smooth and one
  of E_edge, so an undirected mesh edge contributes from both ends with the
  factors s_ij/|N_i| and s_ij/|N_j|.
* s_ij is the mean of the two vertices' non-rigidity weights (Sec. 3.1).
* V^S is the stage's rest geometry: the skinned mesh of the pose stage, or
  the template when the pose stage is not run.  Vh is the rest template.
* Temporal history: with no previous frame both temporal terms are off; with
  one previous frame V^{t-2} is taken equal to V^{t-1}.
* An edge of zero current length has a zero E_edge Jacobian row (its unit
  direction is undefined); the residual still counts in the energy.
* The data terms are those of the embedded-graph stage (module
  ``nonrigid``): bilinear sampling with clamp to edge, central-difference
  image gradients, visibility V and contour set B fixed per frame from the
  exact-arithmetic module, b_i re-evaluated at each linearisation; the
  robust colour kernel sigma_c, the photometric pyramid (module
  ``pyramid``, one Gauss-Newton iteration per level) and the body-part mask
  of the silhouette term (module ``parts``) as there.
* Unknowns update additively, V <- V + delta (no damping, no line search).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp

from . import nonrigid as _nr
from . import parts as _parts
from . import pyramid as _pyr


# ----------------------------------------------------------------------------
# Mesh neighbourhoods
# ----------------------------------------------------------------------------
def one_ring(N: int, tris: np.ndarray):
    """One-ring CSR of a triangle mesh: (off (N+1), dst), each vertex's
    neighbours ascending and unique."""
    F = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    a = np.concatenate([F[:, 0], F[:, 1], F[:, 2], F[:, 1], F[:, 2], F[:, 0]])
    b = np.concatenate([F[:, 1], F[:, 2], F[:, 0], F[:, 0], F[:, 1], F[:, 2]])
    pairs = np.unique(np.stack([a, b], 1), axis=0)          # sorted by (a, b)
    off = np.zeros(N + 1, dtype=np.int64)
    np.add.at(off, pairs[:, 0] + 1, 1)
    return np.cumsum(off), pairs[:, 1].copy()


def pair_sources(off: np.ndarray) -> np.ndarray:
    """Source vertex of every CSR entry."""
    return np.repeat(np.arange(len(off) - 1), np.diff(off))


# ----------------------------------------------------------------------------
# Problem data
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class SurfaceProblem:
    base: np.ndarray        # (N,3) V^S
    tpl: np.ndarray         # (N,3) rest template Vh
    albedo: np.ndarray      # (N,3)
    material: np.ndarray    # (N,) non-rigidity weights
    tris: np.ndarray        # (T,3)
    f: float
    cx: float
    cy: float
    W: int
    H: int
    rgb: np.ndarray
    dt: np.ndarray
    mask: np.ndarray
    w_photo: float
    w_sil: float
    w_smooth: float
    w_edge: float
    w_vel: float
    w_acc: float
    prev1: Optional[np.ndarray] = None   # V^{t-1}
    prev2: Optional[np.ndarray] = None   # V^{t-2}
    vis: Optional[np.ndarray] = None
    inB: Optional[np.ndarray] = None
    bsign: Optional[np.ndarray] = None
    sigma_c: float = 0.0                 # robust colour kernel threshold (0: off)
    pruned: Optional[np.ndarray] = None  # (N,) given pruning decisions (None: decide here)
    pyr_levels: int = 0                  # photometric pyramid levels (0: raw image)
    pyr_ksize: tuple = _pyr.DEFAULT_KSIZE
    level: Optional[int] = None          # pyramid level sampled now (None: raw image)
    part_mask: Optional[np.ndarray] = None   # (H,W) uint8 body-part mask of V^S (None: off)
    vpart: Optional[np.ndarray] = None       # (N,) uint8 part of every vertex

    def __post_init__(self):
        f64 = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
        self.base, self.tpl, self.albedo = f64(self.base), f64(self.tpl), f64(self.albedo)
        self.material, self.rgb, self.dt = f64(self.material), f64(self.rgb), f64(self.dt)
        self.tris = np.asarray(self.tris, dtype=np.int32)
        self.off, self.dst = one_ring(len(self.base), self.tris)
        self.src = pair_sources(self.off)
        deg = np.diff(self.off).astype(np.float64)
        self.s = 0.5 * (self.material[self.src] + self.material[self.dst])
        self.s_over_deg = self.s / deg[self.src]                     # s_ij / |N_i|
        self.rest_len = np.linalg.norm(self.tpl[self.src] - self.tpl[self.dst], axis=1)
        self._grads = None

    @property
    def N(self) -> int:
        return len(self.base)

    def history(self):
        """(w_v, w_a, V^{t-1}, V^{t-2}) after the history reading."""
        if self.prev1 is None:
            return 0.0, 0.0, None, None
        p1 = np.asarray(self.prev1, dtype=np.float64)
        p2 = p1 if self.prev2 is None else np.asarray(self.prev2, dtype=np.float64)
        return self.w_vel, self.w_acc, p1, p2

    def grads(self):
        if self._grads is None:
            self._grads = (_nr.central_differences(self.rgb), _nr.central_differences(self.dt))
        return self._grads


# ----------------------------------------------------------------------------
# Residuals
# ----------------------------------------------------------------------------
def residuals(P: SurfaceProblem, V: np.ndarray) -> dict:
    """All residual blocks at vertex positions V (N,3)."""
    V = np.asarray(V, dtype=np.float64)
    u, w, valid, inimg = _nr.project(P, V)
    photo_on = _nr.prune(P, inimg & P.vis, u, w)
    sil_on = inimg & P.inB & ~_parts.masked(P, V)
    photo = np.zeros((P.N, 3))
    sil = np.zeros(P.N)
    if photo_on.any():
        photo[photo_on] = np.sqrt(P.w_photo) * (_nr.photo_sample(P, u[photo_on], w[photo_on])
                                                - P.albedo[photo_on])
    if sil_on.any():
        sil[sil_on] = np.sqrt(P.w_sil) * _nr.bilinear(P.dt, u[sil_on], w[sil_on])
    d = V[P.src] - V[P.dst]
    dS = P.base[P.src] - P.base[P.dst]
    smooth = np.sqrt(P.w_smooth * P.s_over_deg)[:, None] * (d - dS)
    edge = np.sqrt(P.w_edge * P.s_over_deg) * (np.linalg.norm(d, axis=1) - P.rest_len)
    wv, wa, p1, p2 = P.history()
    vel = np.sqrt(wv) * (V - p1) if p1 is not None else np.zeros((P.N, 3))
    acc = np.sqrt(wa) * (V - 2.0 * p1 + p2) if p1 is not None else np.zeros((P.N, 3))
    return dict(u=u, w=w, photo=photo, sil=sil, photo_on=photo_on, sil_on=sil_on,
                smooth=smooth, edge=edge, vel=vel, acc=acc)


def energy(P: SurfaceProblem, V: np.ndarray) -> dict:
    r = residuals(P, V)
    e = dict(photo=float((r["photo"] ** 2).sum()), sil=float((r["sil"] ** 2).sum()),
             smooth=float((r["smooth"] ** 2).sum()), edge=float((r["edge"] ** 2).sum()),
             velocity=float((r["vel"] ** 2).sum()), acceleration=float((r["acc"] ** 2).sum()))
    e["total"] = sum(e.values())
    return e


def update_directions(P: SurfaceProblem, V: np.ndarray):
    """b_i of the frame's contour set at the current FP32 surface."""
    if P.inB is None:
        return
    from . import visibility as _vis
    neg = _vis.directions(np.asarray(V, dtype=np.float32), P.tris, P.f, P.cx, P.cy, P.W, P.H,
                          P.dt.astype(np.float32), P.mask, P.inB)
    P.bsign = np.where(neg, -1.0, 1.0)


def frame_decisions(P: SurfaceProblem, V: np.ndarray, eps=1e-2):
    """Visibility, B and b_i at the FP32 positions V (the frame's start)."""
    from . import visibility as _vis
    out = _vis.visibility(np.asarray(V, dtype=np.float32), P.tris, P.f, P.cx, P.cy, P.W, P.H,
                          P.dt.astype(np.float32), P.mask, eps)
    fl = out["flags"]
    P.vis = (fl & _vis.FLAG_VISIBLE) != 0
    P.inB = (fl & _vis.FLAG_INB) != 0
    P.bsign = np.where((fl & _vis.FLAG_BNEG) != 0, -1.0, 1.0)
    return out


# ----------------------------------------------------------------------------
# Jacobian
# ----------------------------------------------------------------------------
def linearise(P: SurfaceProblem, V: np.ndarray, directions: bool = True):
    """Stacked residual vector F and its sparse FP64 Jacobian J (columns
    3i..3i+2 = vertex i).  Row blocks: photometric, silhouette, smooth,
    edge, velocity, acceleration."""
    V = np.asarray(V, dtype=np.float64)
    N = P.N
    if directions:
        update_directions(P, V)
    r = residuals(P, V)
    u, w = r["u"], r["w"]
    gxD, gyD = P.grads()[1]
    Dp = _nr.dproj(P, V)
    rows, cols, vals, Fs = [], [], [], []
    row0 = 0

    def block(rr, cc, vv):
        rows.append(np.broadcast_to(rr, vv.shape).ravel())
        cols.append(np.broadcast_to(cc, vv.shape).ravel())
        vals.append(vv.ravel())

    ip = np.nonzero(r["photo_on"])[0]
    if len(ip):
        G = _nr.photo_sample(P, u[ip], w[ip], grad=True)[1]               # (m,3,2)
        A = np.sqrt(P.w_photo) * (G @ Dp[ip])                          # (m,3,3)
        block(row0 + 3 * np.arange(len(ip))[:, None, None] + np.arange(3)[None, :, None],
              3 * ip[:, None, None] + np.arange(3)[None, None, :], A)
        Fs.append(r["photo"][ip].ravel())
        row0 += 3 * len(ip)
    isl = np.nonzero(r["sil_on"])[0]
    if len(isl):
        G = np.stack([_nr.bilinear(gxD, u[isl], w[isl]), _nr.bilinear(gyD, u[isl], w[isl])], axis=1)
        A = (np.sqrt(P.w_sil) * P.bsign[isl])[:, None] * np.einsum("mk,mkj->mj", G, Dp[isl])
        block(row0 + np.arange(len(isl))[:, None], 3 * isl[:, None] + np.arange(3)[None, :], A)
        Fs.append(r["sil"][isl])
        row0 += len(isl)
    npair = len(P.src)
    if npair:
        c = np.sqrt(P.w_smooth * P.s_over_deg)
        I3 = np.broadcast_to(np.eye(3), (npair, 3, 3)) * c[:, None, None]
        rr = row0 + 3 * np.arange(npair)[:, None, None] + np.arange(3)[None, :, None]
        block(rr, 3 * P.src[:, None, None] + np.arange(3)[None, None, :], I3)
        block(rr, 3 * P.dst[:, None, None] + np.arange(3)[None, None, :], -I3)
        Fs.append(r["smooth"].ravel())
        row0 += 3 * npair
        d = V[P.src] - V[P.dst]
        L = np.linalg.norm(d, axis=1)
        n = np.where(L[:, None] > 0.0, d / np.where(L > 0.0, L, 1.0)[:, None], 0.0)
        ce = np.sqrt(P.w_edge * P.s_over_deg)[:, None] * n
        rr = row0 + np.arange(npair)[:, None]
        block(rr, 3 * P.src[:, None] + np.arange(3)[None, :], ce)
        block(rr, 3 * P.dst[:, None] + np.arange(3)[None, :], -ce)
        Fs.append(r["edge"])
        row0 += npair
    wv, wa, p1, _ = P.history()
    if p1 is not None:
        for wt, key in ((wv, "vel"), (wa, "acc")):
            rr = row0 + 3 * np.arange(N)[:, None] + np.arange(3)[None, :]
            block(rr, 3 * np.arange(N)[:, None] + np.arange(3)[None, :],
                  np.full((N, 3), np.sqrt(wt)))
            Fs.append(r[key].ravel())
            row0 += 3 * N
    Fv = np.concatenate(Fs) if Fs else np.zeros(0)
    if rows:
        J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(row0, 3 * N)).tocsr()
    else:
        J = sp.csr_matrix((0, 3 * N))
    return Fv, J


def normal_equations(P: SurfaceProblem, V: np.ndarray, directions: bool = True):
    """(J^T J, -J^T F, F, J) at V."""
    F, J = linearise(P, V, directions)
    JT = J.T.tocsr()
    return (JT @ J).tocsr(), -(JT @ F), F, J


def gauss_newton(P: SurfaceProblem, V: np.ndarray, n_gn: int, n_pcg: int):
    """Fixed-count Gauss-Newton over the vertex positions (no damping)."""
    V = np.asarray(V, dtype=np.float64).copy()
    hist = []
    for gn in range(n_gn):
        P.level = _pyr.level_of(gn, P.pyr_levels)
        A, b, F, _ = normal_equations(P, V)
        delta, info = _nr.pcg(A, b, n_pcg)
        hist.append(dict(energy=float(F @ F), step_norm=float(np.linalg.norm(delta)),
                         pcg_iters=info["iters"], breakdown=info["breakdown"]))
        V = V + delta.reshape(-1, 3)
    P.level = _nr.final_level(P)
    return V, hist


# ----------------------------------------------------------------------------
# Displacement warping (Sec. 3.4)
# ----------------------------------------------------------------------------
def blend_rotations(G: np.ndarray, skin_idx: np.ndarray, skin_w: np.ndarray) -> np.ndarray:
    """Per-vertex rotation of the dual-quaternion blend of the bone
    rotations G (J,3,3) with the skinning weights (N,S): the bones'
    quaternions, each sign-aligned with the quaternion of the vertex's first
    bone, summed with the weights and normalised (the rotation part of dual
    quaternion skinning).  Returns (N,3,3); the identity where the sum is 0."""
    from scipy.spatial.transform import Rotation
    q = Rotation.from_matrix(np.asarray(G, dtype=np.float64)).as_quat()      # (J,4) x, y, z, w
    idx = np.asarray(skin_idx, dtype=np.int64)
    w = np.asarray(skin_w, dtype=np.float64)
    qs = q[idx]                                                               # (N,S,4)
    sign = np.where(np.einsum("nsk,nk->ns", qs, qs[:, 0]) < 0.0, -1.0, 1.0)
    blend = np.einsum("ns,nsk->nk", w * sign, qs)
    norm = np.linalg.norm(blend, axis=1)
    out = np.tile(np.eye(3), (len(blend), 1, 1))
    ok = norm > 0.0
    if ok.any():
        out[ok] = Rotation.from_quat(blend[ok] / norm[ok, None]).as_matrix()
    return out


def record_displacement(V: np.ndarray, VS: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """Rest-pose displacement dh_i = Q_i^T (V_i - V^S_i)."""
    return np.einsum("nji,nj->ni", Q, np.asarray(V, np.float64) - np.asarray(VS, np.float64))


def warped_start(VS: np.ndarray, Q: np.ndarray, dh: np.ndarray) -> np.ndarray:
    """Start of the next frame: V_i = V^S_i + Q_i dh_i."""
    return np.asarray(VS, np.float64) + np.einsum("nij,nj->ni", Q, dh)


def graph_rest_params(R: np.ndarray, t: np.ndarray, node_vid: np.ndarray, Q: np.ndarray):
    """The graph counterpart of the displacement warping: node k's
    parameters carried to the rest pose through the blend rotation
    Q_k = Q[node_vid[k]] of its node vertex, R^rest = Q_k^T R_k Q_k and
    t^rest = Q_k^T t_k.  R (n,3,3) or (n,9), t (n,3)."""
    Qk = np.asarray(Q, dtype=np.float64)[np.asarray(node_vid, dtype=np.int64)]
    Rn = np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)
    return (np.einsum("nji,njk,nkl->nil", Qk, Rn, Qk),
            np.einsum("nji,nj->ni", Qk, np.asarray(t, dtype=np.float64).reshape(-1, 3)))


def graph_posed_params(R_rest: np.ndarray, t_rest: np.ndarray, node_vid: np.ndarray, Q: np.ndarray):
    """Rest-pose node parameters posed with the blend rotations Q of a new
    pose: R_k = Q_k R^rest_k Q_k^T, t_k = Q_k t^rest_k."""
    Qk = np.asarray(Q, dtype=np.float64)[np.asarray(node_vid, dtype=np.int64)]
    return (np.einsum("nij,njk,nlk->nil", Qk, np.asarray(R_rest, dtype=np.float64), Qk),
            np.einsum("nij,nj->ni", Qk, np.asarray(t_rest, dtype=np.float64)))


# ----------------------------------------------------------------------------
# Assembling a problem from scene data
# ----------------------------------------------------------------------------
def problem_from_scene(scene, base32: Optional[np.ndarray] = None, weights=None,
                       prev1=None, prev2=None) -> SurfaceProblem:
    """Problem for a scene (``synth.Scene``): ``base32`` is V^S (default: the
    template); ``weights`` = (w_photo, w_sil, w_smooth, w_edge, w_vel, w_acc),
    default the scene's surface weights."""
    base = np.asarray(scene.V if base32 is None else base32, dtype=np.float32)
    wp, ws, wsm, wed, wv, wa = scene.surface_weights if weights is None else weights
    return SurfaceProblem(
        base=base, tpl=scene.V, albedo=scene.albedo, material=scene.material, tris=scene.F,
        f=float(np.float32(scene.cam.f)), cx=float(np.float32(scene.cam.cx)),
        cy=float(np.float32(scene.cam.cy)), W=scene.cam.W, H=scene.cam.H,
        rgb=scene.rgb, dt=scene.dt, mask=scene.mask,
        w_photo=wp, w_sil=ws, w_smooth=wsm, w_edge=wed, w_vel=wv, w_acc=wa,
        prev1=prev1, prev2=prev2)


def solve_scene(scene, base32=None, V0=None, n_gn=None, n_pcg=None, prev1=None, prev2=None,
                sigma_c: float = 0.0, pyr_levels: int = 0, pyr_ksize=_pyr.DEFAULT_KSIZE,
                part_mask=None, vpart=None):
    """Whole surface solve of one frame: decisions at the FP32 start V0
    (default V^S), then n_gn x n_pcg Gauss-Newton (``sigma_c``, the robust
    colour kernel's threshold, 0 = off; ``pyr_levels``, the photometric
    pyramid's levels, 0 = raw image; ``part_mask`` / ``vpart``, the body-part
    mask of the silhouette term, None = off).  Returns a dict."""
    P = problem_from_scene(scene, base32, prev1=prev1, prev2=prev2)
    P.sigma_c = float(sigma_c)
    P.pyr_levels, P.pyr_ksize = int(pyr_levels), tuple(pyr_ksize)
    P.part_mask, P.vpart = part_mask, vpart
    V = P.base.copy() if V0 is None else np.asarray(V0, dtype=np.float32).astype(np.float64)
    frame_decisions(P, V.astype(np.float32))
    P.level = _pyr.level_of(0, P.pyr_levels)
    e0 = energy(P, V)
    V, hist = gauss_newton(P, V, scene.n_gn_surface if n_gn is None else n_gn,
                           scene.n_pcg_surface if n_pcg is None else n_pcg)
    return dict(problem=P, V=V, hist=hist, e0=e0, e1=energy(P, V))
