"""Skeletal pose stage in FP64 (Sec. 3.3 and Sec. 4, pose estimation).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Energy:
    E_pose = lambda_2D sum_j ||pi(o_j) - P2D_j||^2            (2D joints, pixels)
           + lambda_3D sum_j ||o_j - P3D_j||^2                (3D joints, metres)
           + lambda_sil/|B| sum_{i in B} I_DT(pi(V^S_i))^2     (silhouette, b_i sign)
           + lambda_temporal sum_j w_j ||o_j - o_j^{t-1}||^2   (temporal stabilisation)
           + lambda_anatomic sum_{Euler DOF} Psi(theta)        (joint angle limits)
           + lambda_prior sum_{Euler DOF} (theta - theta_init)^2
over the pose vector [root axis-angle (3), root translation (3), Euler XYZ
angles of every DOF joint (3 each)].

Readings:
* Forward kinematics: o_root = t, G_root = R_root; for a child j of p,
  o_j = o_p + G_p (J_j - J_p) with rest joint positions J, G_j = G_p L_j,
  L_j = Rx(a) Ry(b) Rz(c) for a DOF joint and I for an end site.
* Linear blend skinning of the rest template:
  V^S_i = sum_b w_ib (G_b (V_i - J_b) + o_b).
* The root rotation is updated on the left, R <- Exp(d_omega) R, the
  translation and Euler angles additively (Gauss-Newton, Sec. 4).
* The 3D joint term uses global 3D detections, so the paper's auxiliary
  translation t' and bone-length rescaling are not needed.
* The angle prior (lambda_prior, default 1e4) keeps the normal matrix
  positive definite and undamped Gauss-Newton stable: twists about a bone
  whose only child lies on the bone axis move no joint and, on rotationally
  symmetric capsule limbs, no silhouette, and the hand / head segments are
  short, so noisy detections otherwise drive radian-sized steps.  It plays
  the role of the paper's temporal term in angle space.
* The silhouette weight is divided by |B| so that the term does not grow
  with the mesh resolution (the paper gives no units for its weights).
* The contour set B comes from the skinned mesh at the frame's initial pose
  (once per frame, Sec. 3.3); b_i is re-evaluated on the current skinned
  surface at every linearisation.  Both through the exact visibility module.
* E_temporal (Sec. 3.3) compares the joints with the previous frame's; it
  is off until a previous frame has been recorded.  E_anatomic's barrier
  Psi(x) = (x - max)^2 above the limit, (min - x)^2 below, 0 inside, enters
  Gauss-Newton as a residual sqrt(lambda)(theta - bound) on the DOFs outside
  their limits at the linearisation point (no limits: off).
* Frame start (Sec. 3.3): an explicit Euler step in angle space from the
  last two frames, theta = 2 theta^{t-1} - theta^{t-2} for the Euler angles
  and the root translation; the root rotation takes the same
  constant-velocity step on SO(3), R = R^{t-1} (R^{t-2})^T R^{t-1}.
* Skinned displacement (Sec. 3.4, displacement warping): the previous
  frame's rest-pose displacement, carried by the dual-quaternion blend
  rotation of the frame's start pose, d^S = Q(theta_start) dhat, is added to
  the skinned model for the silhouette term and the frame decisions.  Reading:
  it is held fixed during the pose solve (the paper does not say how it
  enters the Jacobian), so the Jacobian is the skinning's.
* The normal equations are solved by a Cholesky factorisation (FP64).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from . import nonrigid as nr


def euler_xyz(a: np.ndarray) -> np.ndarray:
    """Rx(a0) Ry(a1) Rz(a2) for rows of a (m,3) -> (m,3,3)."""
    a = np.atleast_2d(a)
    c, s = np.cos(a), np.sin(a)
    one, zero = np.ones(len(a)), np.zeros(len(a))
    Rx = np.stack([np.stack([one, zero, zero], -1), np.stack([zero, c[:, 0], -s[:, 0]], -1),
                   np.stack([zero, s[:, 0], c[:, 0]], -1)], -2)
    Ry = np.stack([np.stack([c[:, 1], zero, s[:, 1]], -1), np.stack([zero, one, zero], -1),
                   np.stack([-s[:, 1], zero, c[:, 1]], -1)], -2)
    Rz = np.stack([np.stack([c[:, 2], -s[:, 2], zero], -1), np.stack([s[:, 2], c[:, 2], zero], -1),
                   np.stack([zero, zero, one], -1)], -2)
    return Rx @ Ry @ Rz


@dataclasses.dataclass
class Skeleton:
    parents: np.ndarray        # (J,)
    joints_rest: np.ndarray    # (J,3)
    dof: np.ndarray            # (J,) bool: ball joint (root: always 6 DOF)
    skin_idx: np.ndarray       # (N,4)
    skin_w: np.ndarray         # (N,4)

    def __post_init__(self):
        self.parents = np.asarray(self.parents, dtype=np.int64)
        self.joints_rest = np.asarray(self.joints_rest, dtype=np.float64)
        self.dof = np.asarray(self.dof, dtype=bool)
        self.skin_idx = np.asarray(self.skin_idx, dtype=np.int64)
        self.skin_w = np.asarray(self.skin_w, dtype=np.float64)
        J = len(self.parents)
        # column offset of each DOF joint's Euler angles in the pose vector
        self.col = np.full(J, -1, dtype=np.int64)
        c = 6
        for j in range(1, J):
            if self.dof[j]:
                self.col[j] = c
                c += 3
        self.n_dof = c
        # ancestors (including the joint itself)
        self.anc = np.zeros((J, J), dtype=bool)
        for j in range(J):
            a = j
            while a >= 0:
                self.anc[j, a] = True
                a = self.parents[a]


def skeleton_from_scene(scene) -> Skeleton:
    sk = scene.skeleton
    dof = np.ones(len(sk["parents"]), dtype=bool)
    from synth.scenes import SKELETON_SITES
    dof[SKELETON_SITES] = False
    dof[0] = True
    return Skeleton(sk["parents"], sk["joints_rest"], dof, sk["skin_idx"], sk["skin_w"])


def split_pose(sk: Skeleton, pose: np.ndarray):
    pose = np.asarray(pose, dtype=np.float64)
    R_root = nr.so3_exp(pose[:3])[0]
    t_root = pose[3:6].copy()
    ang = np.zeros((len(sk.parents), 3))
    for j in range(1, len(sk.parents)):
        if sk.dof[j]:
            ang[j] = pose[sk.col[j]:sk.col[j] + 3]
    return R_root, t_root, ang


def forward_kinematics(sk: Skeleton, R_root, t_root, ang):
    """Global joint rotations G (J,3,3) and positions o (J,3)."""
    J = len(sk.parents)
    G = np.zeros((J, 3, 3))
    o = np.zeros((J, 3))
    L = euler_xyz(ang)
    for j in range(J):
        p = sk.parents[j]
        if p < 0:
            G[j] = R_root
            o[j] = t_root
        else:
            o[j] = o[p] + G[p] @ (sk.joints_rest[j] - sk.joints_rest[p])
            G[j] = G[p] @ (L[j] if sk.dof[j] else np.eye(3))
    return G, o


def skin(sk: Skeleton, V: np.ndarray, G, o):
    """Per-slot bone transforms P (N,4,3) and the skinned positions (N,3)."""
    b = sk.skin_idx
    P = np.einsum("nsij,nsj->nsi", G[b], V[:, None, :] - sk.joints_rest[b]) + o[b]
    return P, np.einsum("ns,nsi->ni", sk.skin_w, P)


def joint_axes(sk: Skeleton, G, ang):
    """World rotation axes (J,3,3) of the Euler angles a, b, c of each joint:
    u_a = G_p e_x, u_b = G_p Rx(a) e_y, u_c = G_p Rx(a) Ry(b) e_z."""
    J = len(sk.parents)
    U = np.zeros((J, 3, 3))
    for j in range(1, J):
        if not sk.dof[j]:
            continue
        Gp = G[sk.parents[j]]
        a, bb = ang[j, 0], ang[j, 1]
        Rx = euler_xyz(np.array([[a, 0.0, 0.0]]))[0]
        Ry = euler_xyz(np.array([[0.0, bb, 0.0]]))[0]
        U[j, 0] = Gp[:, 0]
        U[j, 1] = Gp @ Rx[:, 1]
        U[j, 2] = Gp @ (Rx @ Ry)[:, 2]
    return U


def point_jacobian(sk: Skeleton, P, owner_bones, t_root, o, U):
    """d P / d pose for points P (m,3) rigidly attached to bone owner_bones[m]:
    (m,3,n_dof).  Root: -[P - t]x (left rotation), I; joint j's Euler axis u
    moves P by u x (P - o_j) if j is an ancestor of the owning bone."""
    m = len(P)
    Jp = np.zeros((m, 3, sk.n_dof))
    Jp[:, :, 0:3] = -nr.hat(P - t_root)
    Jp[:, :, 3:6] = np.eye(3)
    for j in range(1, len(sk.parents)):
        if not sk.dof[j]:
            continue
        on = sk.anc[owner_bones, j]
        if not on.any():
            continue
        rel = P[on] - o[j]
        for ax in range(3):
            Jp[on, :, sk.col[j] + ax] = np.cross(U[j, ax][None, :], rel)
    return Jp


@dataclasses.dataclass
class PoseProblem:
    sk: Skeleton
    V: np.ndarray               # (N,3) rest template
    tris: np.ndarray
    f: float
    cx: float
    cy: float
    W: int
    H: int
    dt: np.ndarray
    mask: np.ndarray
    j2d: np.ndarray             # (J,2)
    j3d: np.ndarray             # (J,3)
    lam_2d: float = 460.0
    lam_3d: float = 28.0
    lam_sil: float = 200.0
    lam_prior: float = 1e4
    pose_init: Optional[np.ndarray] = None
    lam_temporal: float = 1.5
    temporal_w: Optional[np.ndarray] = None    # (J,) per-joint weights, default 1
    prev_joints: Optional[np.ndarray] = None   # (J,3) joints of the previous frame
    lam_anatomic: float = 1e6
    theta_min: Optional[np.ndarray] = None     # (n_dof,) limits, -inf / +inf where none
    theta_max: Optional[np.ndarray] = None
    inB: Optional[np.ndarray] = None
    bsign: Optional[np.ndarray] = None
    disp: Optional[np.ndarray] = None          # (N,3) skinned displacement d^S added to the skinned model

    def __post_init__(self):
        self.V = np.asarray(self.V, dtype=np.float64)
        self.dt = np.asarray(self.dt, dtype=np.float64)
        self.j2d = np.asarray(self.j2d, dtype=np.float64)
        self.j3d = np.asarray(self.j3d, dtype=np.float64)
        self._gdt = None

    def gdt(self):
        if self._gdt is None:
            self._gdt = nr.central_differences(self.dt)
        return self._gdt


def _proj(pb: PoseProblem, X):
    Z = X[:, 2]
    ok = Z > 1e-3
    Zs = np.where(ok, Z, 1.0)
    u = pb.f * X[:, 0] / Zs + pb.cx
    v = pb.f * X[:, 1] / Zs + pb.cy
    D = np.zeros((len(X), 2, 3))
    D[:, 0, 0] = pb.f / Zs
    D[:, 0, 2] = -pb.f * X[:, 0] / (Zs * Zs)
    D[:, 1, 1] = pb.f / Zs
    D[:, 1, 2] = -pb.f * X[:, 1] / (Zs * Zs)
    inimg = ok & (u >= 0) & (u <= pb.W - 1) & (v >= 0) & (v <= pb.H - 1)
    return u, v, D, ok, inimg


def residuals_and_jacobian(pb: PoseProblem, pose: np.ndarray):
    """Stacked residual F and dense Jacobian J (rows x n_dof), FP64.

    Rows: 2D joints (2 per joint, joints with Z > 1e-3), 3D joints (3 per
    joint), silhouette (1 per contour vertex inside the image, weight
    lambda_sil / |B|, Jacobian row times b_i), angle prior (1 per Euler
    DOF)."""
    sk = pb.sk
    R, t, ang = split_pose(sk, pose)
    G, o = forward_kinematics(sk, R, t, ang)
    U = joint_axes(sk, G, ang)
    Jn = len(sk.parents)
    Jo = point_jacobian(sk, o, np.arange(Jn), t, o, U)   # joints ride on themselves
    rows, Fs = [], []
    u, v, D, ok, _ = _proj(pb, o)
    s2 = np.sqrt(pb.lam_2d)
    for j in np.nonzero(ok)[0]:
        Fs.append(s2 * (np.array([u[j], v[j]]) - pb.j2d[j]))
        rows.append(s2 * (D[j] @ Jo[j]))
    s3 = np.sqrt(pb.lam_3d)
    Fs.append(s3 * (o - pb.j3d).ravel())
    rows.append(s3 * Jo.reshape(-1, sk.n_dof))
    if pb.inB is not None and pb.inB.any():
        P, VS = skin(sk, pb.V, G, o)
        if pb.disp is not None:
            VS = VS + pb.disp      # held fixed over the solve: the Jacobian is the skinning's
        # b_i follows the current skinned surface (the contour set B does not);
        # with no triangles given the caller's b_i stay fixed
        if pb.tris is not None:
            from . import visibility as _vis
            neg = _vis.directions(VS.astype(np.float32), pb.tris, pb.f, pb.cx, pb.cy, pb.W, pb.H,
                                  pb.dt.astype(np.float32), pb.mask, pb.inB)
            pb.bsign = np.where(neg, -1.0, 1.0)
        uu, vv, DD, okv, inimg = _proj(pb, VS)
        sel = np.nonzero(pb.inB & inimg)[0]
        if len(sel):
            gx, gy = pb.gdt()
            ss = np.sqrt(pb.lam_sil / max(1, int(pb.inB.sum())))
            Fs.append(ss * nr.bilinear(pb.dt, uu[sel], vv[sel]))
            g = np.stack([nr.bilinear(gx, uu[sel], vv[sel]), nr.bilinear(gy, uu[sel], vv[sel])], 1)
            # d V^S / d pose = sum_s w_s d P_s / d pose
            Jv = np.zeros((len(sel), 3, sk.n_dof))
            for sl in range(sk.skin_idx.shape[1]):
                bones = sk.skin_idx[sel, sl]
                Jv += sk.skin_w[sel, sl, None, None] * point_jacobian(sk, P[sel, sl], bones, t, o, U)
            Jr = np.einsum("mk,mkd->md", g, np.einsum("mkc,mcd->mkd", DD[sel], Jv))
            rows.append((ss * pb.bsign[sel])[:, None] * Jr)
    if pb.prev_joints is not None and pb.lam_temporal > 0:
        w = np.ones(Jn) if pb.temporal_w is None else np.asarray(pb.temporal_w, dtype=np.float64)
        st = np.sqrt(pb.lam_temporal * w)
        Fs.append((st[:, None] * (o - np.asarray(pb.prev_joints, dtype=np.float64))).ravel())
        rows.append((st[:, None, None] * Jo).reshape(-1, sk.n_dof))
    if pb.theta_min is not None and pb.lam_anatomic > 0:
        th = np.asarray(pose, dtype=np.float64)
        lo = np.asarray(pb.theta_min, dtype=np.float64)
        hi = np.asarray(pb.theta_max, dtype=np.float64)
        sa = np.sqrt(pb.lam_anatomic)
        for c in range(6, sk.n_dof):
            bound = hi[c] if th[c] > hi[c] else (lo[c] if th[c] < lo[c] else None)
            if bound is None:
                continue
            Fs.append(np.array([sa * (th[c] - bound)]))
            r = np.zeros(sk.n_dof)
            r[c] = sa
            rows.append(r[None])
    if pb.lam_prior > 0:
        sp = np.sqrt(pb.lam_prior)
        base = pb.pose_init if pb.pose_init is not None else np.zeros(sk.n_dof)
        Fp = sp * (np.asarray(pose)[6:] - base[6:])
        Jp = np.zeros((sk.n_dof - 6, sk.n_dof))
        Jp[:, 6:] = sp * np.eye(sk.n_dof - 6)
        Fs.append(Fp)
        rows.append(Jp)
    F = np.concatenate([np.atleast_1d(np.asarray(f, dtype=np.float64)).ravel() for f in Fs])
    Jm = np.concatenate([np.atleast_2d(r).reshape(-1, sk.n_dof) for r in rows])
    return F, Jm


def cholesky_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Plain Cholesky A = L L^T (raises on a non-positive pivot), then two
    triangular solves."""
    n = len(A)
    L = np.zeros_like(A)
    for j in range(n):
        d = A[j, j] - L[j, :j] @ L[j, :j]
        if not d > 0.0:
            raise np.linalg.LinAlgError("non-positive pivot")
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    x = np.zeros(n)
    for i in reversed(range(n)):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def apply_update(sk: Skeleton, pose: np.ndarray, delta: np.ndarray) -> np.ndarray:
    out = np.asarray(pose, dtype=np.float64).copy()
    R = nr.so3_exp(delta[:3])[0] @ nr.so3_exp(out[:3])[0]
    out[:3] = nr.so3_log(R)[0]
    out[3:] += delta[3:]
    return out


def energy(pb: PoseProblem, pose) -> float:
    F, _ = residuals_and_jacobian(pb, pose)
    return float(F @ F)


def frame_decisions(pb: PoseProblem, pose):
    """B and b_i on the skinned mesh at `pose` (FP64 skinning rounded to FP32,
    then the exact module)."""
    from . import visibility as _vis
    R, t, ang = split_pose(pb.sk, pose)
    G, o = forward_kinematics(pb.sk, R, t, ang)
    _, VS = skin(pb.sk, pb.V, G, o)
    if pb.disp is not None:
        VS = VS + pb.disp
    out = _vis.visibility(VS.astype(np.float32), pb.tris, pb.f, pb.cx, pb.cy, pb.W, pb.H,
                          pb.dt.astype(np.float32), pb.mask, 1e-2)
    fl = out["flags"]
    pb.inB = (fl & _vis.FLAG_INB) != 0
    pb.bsign = np.where((fl & _vis.FLAG_BNEG) != 0, -1.0, 1.0)
    return out


def gauss_newton(pb: PoseProblem, pose0, n_gn: int):
    pose = np.asarray(pose0, dtype=np.float64).copy()
    hist = []
    for _ in range(n_gn):
        F, J = residuals_and_jacobian(pb, pose)
        A = J.T @ J
        g = -(J.T @ F)
        delta = cholesky_solve(A, g)
        hist.append(dict(energy=float(F @ F), step_norm=float(np.linalg.norm(delta))))
        pose = apply_update(pb.sk, pose, delta)
    return pose, hist


def skinned_displacement(sk: Skeleton, pose: np.ndarray, dhat: np.ndarray) -> np.ndarray:
    """d^S = Q(pose) dhat: the rest-pose displacement of the previous frame
    carried by the rotation of the dual-quaternion blend of the bone
    rotations at `pose` (Sec. 3.4, displacement warping)."""
    from .surface import blend_rotations
    R, t, ang = split_pose(sk, pose)
    G, o = forward_kinematics(sk, R, t, ang)
    Q = blend_rotations(G, sk.skin_idx, sk.skin_w)
    return np.einsum("nij,nj->ni", Q, np.asarray(dhat, dtype=np.float64))


def extrapolate(pose1: np.ndarray, pose2: Optional[np.ndarray] = None) -> np.ndarray:
    """Frame start from the last two poses (pose1 = t-1, pose2 = t-2): the
    explicit Euler step of the reading above; pose1 itself without pose2."""
    p1 = np.asarray(pose1, dtype=np.float64)
    if pose2 is None:
        return p1.copy()
    p2 = np.asarray(pose2, dtype=np.float64)
    out = 2.0 * p1 - p2
    R1 = nr.so3_exp(p1[:3])[0]
    R2 = nr.so3_exp(p2[:3])[0]
    out[:3] = nr.so3_log(R1 @ R2.T @ R1)[0]
    return out


def problem_from_scene(scene, lam_prior=1e4) -> PoseProblem:
    sk = skeleton_from_scene(scene)
    return PoseProblem(sk=sk, V=scene.V, tris=scene.F, f=float(np.float32(scene.cam.f)),
                       cx=float(np.float32(scene.cam.cx)), cy=float(np.float32(scene.cam.cy)),
                       W=scene.cam.W, H=scene.cam.H, dt=scene.dt, mask=scene.mask,
                       j2d=scene.joints2d, j3d=scene.joints3d, lam_prior=lam_prior,
                       pose_init=np.asarray(scene.pose_init, dtype=np.float64))


def solve_scene(scene, n_gn: Optional[int] = None, lam_prior=1e4):
    """Pose stage for a body scene from its initial pose.  Returns a dict
    with the final pose, history, skinned vertices (FP64) and joints."""
    pb = problem_from_scene(scene, lam_prior)
    pose0 = np.asarray(scene.pose_init, dtype=np.float64)
    frame_decisions(pb, pose0)
    e0 = energy(pb, pose0)
    pose, hist = gauss_newton(pb, pose0, scene.n_gn_pose if n_gn is None else n_gn)
    R, t, ang = split_pose(pb.sk, pose)
    G, o = forward_kinematics(pb.sk, R, t, ang)
    _, VS = skin(pb.sk, pb.V, G, o)
    return dict(problem=pb, pose=pose, hist=hist, e0=e0, e1=energy(pb, pose), VS=VS, joints=o)
