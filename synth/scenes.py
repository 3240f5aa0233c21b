"""Scene generators: meshes, appearance, skeleton, ground truth, target frames.

Every random draw comes from ``numpy.random.default_rng(seed)`` or, for the
value-noise lattice, from the splitmix64 finaliser applied to lattice
coordinates.  All geometry is produced in FP64 and handed out as FP32 arrays,
which is the precision the library's upload calls take.

Workloads (sizes follow the problem statement of the non-rigid stage,
Sec. 3.4, at the scales of the synthetic configurations):

* ``"tiny"``: closed capsule, 1,002 vertices / 2,000 triangles, 64 nodes, K=4,
  128x128 image, f=150 px.
* ``"body"``: articulated capsule body (10 capsules), 6,020 vertices /
  12,000 triangles, 500 nodes, K=4, 1024x1024 image, 23-joint skeleton.
* ``"stress"``: a body of about 100,000 vertices, 4,000 nodes, K=8, 2048x2048.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np
from scipy import ndimage

# ----------------------------------------------------------------------------
# splitmix64 (Steele, Lea, Flood 2014) — used for the value-noise lattice
# ----------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied element-wise to uint64 states."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def _lattice_value(ix, iy, iz, salt: int) -> np.ndarray:
    """Uniform [0,1) value attached to an integer lattice point."""
    with np.errstate(over="ignore"):
        h = splitmix64(np.uint64(salt) * np.uint64(0x632BE59BD9B4E019))
        h = splitmix64(h ^ ix.astype(np.int64).astype(np.uint64))
        h = splitmix64(h ^ iy.astype(np.int64).astype(np.uint64))
        h = splitmix64(h ^ iz.astype(np.int64).astype(np.uint64))
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------
# Camera
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Camera:
    """Static pinhole camera; camera space is world space (Sec. 3.2).

    Pixel centres sit at integer coordinates; the principal point is the
    image centre, (W-1)/2, (H-1)/2.  No distortion.
    """

    f: float
    W: int
    H: int

    @property
    def cx(self) -> float:
        return (self.W - 1) * 0.5

    @property
    def cy(self) -> float:
        return (self.H - 1) * 0.5


# ----------------------------------------------------------------------------
# Meshes
# ----------------------------------------------------------------------------
def _profile(radius: float, cyl_len: float, rings: int):
    """(rho, y) of ``rings`` rings spaced evenly in arc length pole to pole."""
    quarter = 0.5 * math.pi * radius
    total = 2.0 * quarter + cyl_len
    s = np.arange(1, rings + 1, dtype=np.float64) * (total / (rings + 1))
    rho = np.empty(rings)
    y = np.empty(rings)
    for j, sj in enumerate(s):
        if sj <= quarter:
            phi = sj / radius
            rho[j] = radius * math.sin(phi)
            y[j] = -0.5 * cyl_len - radius * math.cos(phi)
        elif sj <= quarter + cyl_len:
            rho[j] = radius
            y[j] = -0.5 * cyl_len + (sj - quarter)
        else:
            phi = (sj - quarter - cyl_len) / radius
            rho[j] = radius * math.cos(phi)
            y[j] = 0.5 * cyl_len + radius * math.sin(phi)
    return rho, y, 0.5 * cyl_len + radius


def capsule_mesh(radius: float, total_len: float, rings: int, segments: int):
    """Closed capsule along +Y centred at the origin, outward-oriented.

    Returns (V float64 (2+rings*segments, 3), F int64 (2*V-4, 3)).
    ``total_len`` includes both hemispherical caps.
    """
    cyl = total_len - 2.0 * radius
    assert cyl >= 0.0
    rho, y, half = _profile(radius, cyl, rings)
    ang = 2.0 * math.pi * np.arange(segments) / segments
    ring_pts = np.stack(
        [rho[:, None] * np.cos(ang)[None, :],
         np.repeat(y[:, None], segments, axis=1),
         rho[:, None] * np.sin(ang)[None, :]], axis=-1).reshape(-1, 3)
    V = np.concatenate([[[0.0, -half, 0.0]], ring_pts, [[0.0, half, 0.0]]])
    S = segments
    top = 1 + rings * S
    tris = []
    for k in range(S):
        tris.append((0, 1 + k, 1 + (k + 1) % S))
    for j in range(rings - 1):
        a0 = 1 + j * S
        b0 = 1 + (j + 1) * S
        for k in range(S):
            k1 = (k + 1) % S
            tris.append((a0 + k, b0 + k, b0 + k1))
            tris.append((a0 + k, b0 + k1, a0 + k1))
    last = 1 + (rings - 1) * S
    for k in range(S):
        tris.append((last + k, top, last + (k + 1) % S))
    F = np.asarray(tris, dtype=np.int64)
    # orient every triangle outward (normal away from the capsule axis segment)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    axis_pt = np.zeros_like(cen)
    axis_pt[:, 1] = np.clip(cen[:, 1], -0.5 * cyl, 0.5 * cyl)
    flip = np.einsum("ij,ij->i", n, cen - axis_pt) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def _frame_from_axis(d: np.ndarray) -> np.ndarray:
    """Rotation taking +Y to unit direction d (columns: x', y'=d, z')."""
    d = d / np.linalg.norm(d)
    helper = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(d, helper)
    x /= np.linalg.norm(x)
    z = np.cross(x, d)
    return np.stack([x, d, z], axis=1)


# ----------------------------------------------------------------------------
# Skeleton: 23 joints, 5 of them end sites; root 6 DOF + 17 ball joints x 3
# ----------------------------------------------------------------------------
SKELETON_NAMES = [
    "pelvis", "spine", "chest", "neck", "head_top",
    "l_clavicle", "l_shoulder", "l_elbow", "l_wrist", "l_hand_tip",
    "r_clavicle", "r_shoulder", "r_elbow", "r_wrist", "r_hand_tip",
    "l_hip", "l_knee", "l_ankle", "l_toe",
    "r_hip", "r_knee", "r_ankle", "r_toe",
]
SKELETON_PARENTS = np.array(
    [-1, 0, 1, 2, 3,
     2, 5, 6, 7, 8,
     2, 10, 11, 12, 13,
     0, 15, 16, 17,
     0, 19, 20, 21], dtype=np.int32)
SKELETON_SITES = np.array([4, 9, 14, 18, 22])
# body part of every joint's bone: torso 0, head 1, left arm 2, right arm 3,
# left leg 4, right leg 5 (the labels of the silhouette term's part mask)
SKELETON_BONE_PART = np.array(
    [0, 0, 0, 1, 1,
     2, 2, 2, 2, 2,
     3, 3, 3, 3, 3,
     4, 4, 4, 4,
     5, 5, 5, 5], dtype=np.int32)
TORSO_PART = 0
N_POSE_DOF = 57

# Rest joint positions relative to the pelvis.  Camera convention: +Y points
# down in the image, so the head is at negative Y.  T-pose, facing -Z.
_REST_REL = np.array([
    [0.00, 0.00, 0.00],    # pelvis
    [0.00, -0.12, 0.00],   # spine
    [0.00, -0.30, 0.00],   # chest
    [0.00, -0.50, 0.00],   # neck
    [0.00, -0.76, 0.00],   # head_top
    [0.05, -0.46, 0.00],   # l_clavicle
    [0.20, -0.46, 0.00],   # l_shoulder
    [0.50, -0.46, 0.00],   # l_elbow
    [0.76, -0.46, 0.00],   # l_wrist
    [0.88, -0.46, 0.00],   # l_hand_tip
    [-0.05, -0.46, 0.00],  # r_clavicle
    [-0.20, -0.46, 0.00],  # r_shoulder
    [-0.50, -0.46, 0.00],  # r_elbow
    [-0.76, -0.46, 0.00],  # r_wrist
    [-0.88, -0.46, 0.00],  # r_hand_tip
    [0.10, 0.02, 0.00],    # l_hip
    [0.10, 0.47, 0.00],    # l_knee
    [0.10, 0.90, 0.00],    # l_ankle
    [0.10, 0.95, -0.12],   # l_toe
    [-0.10, 0.02, 0.00],   # r_hip
    [-0.10, 0.47, 0.00],   # r_knee
    [-0.10, 0.90, 0.00],   # r_ankle
    [-0.10, 0.95, -0.12],  # r_toe
])

# capsule: (proximal joint, distal joint, radius, bones along the axis, skin(1)/cloth(0))
# bones along the axis: list of (axial fraction where the bone starts, bone id)
_CAPSULES = [
    ("torso", 0, 3, 0.15, [(0.0, 0), (0.3, 1), (0.6, 2)], 0),
    ("head", 3, 4, 0.10, [(0.0, 3)], 1),
    ("l_upper_arm", 6, 7, 0.055, [(0.0, 6)], 0),
    ("l_forearm", 7, 9, 0.045, [(0.0, 7), (0.7, 8)], 1),
    ("r_upper_arm", 11, 12, 0.055, [(0.0, 11)], 0),
    ("r_forearm", 12, 14, 0.045, [(0.0, 12), (0.7, 13)], 1),
    ("l_thigh", 15, 16, 0.075, [(0.0, 15)], 0),
    ("l_shin", 16, 18, 0.06, [(0.0, 16), (0.85, 17)], 1),
    ("r_thigh", 19, 20, 0.075, [(0.0, 19)], 0),
    ("r_shin", 20, 22, 0.06, [(0.0, 20), (0.85, 21)], 1),
]


def body_template(rings: int = 24, segments: int = 25,
                  root=(0.0, -0.05, 3.0)):
    """Articulated capsule body in its rest (T) pose, in world coordinates.

    Returns a dict with V (N,3), F (T,3), per-vertex segment id, skin flag,
    LBS binding (4 bones per vertex: ``skin_idx`` int, ``skin_w`` float, rows
    summing to 1), rest joint positions ``joints_rest`` (23,3) and ``parents``.
    """
    root = np.asarray(root, dtype=np.float64)
    joints = _REST_REL + root
    Vs, Fs, seg, skin, sidx, sw = [], [], [], [], [], []
    base = 0
    for ci, (name, pa, pb, r, bones, is_skin) in enumerate(_CAPSULES):
        A, B = joints[pa], joints[pb]
        L = float(np.linalg.norm(B - A))
        V, F = capsule_mesh(r, L + 2.0 * r, rings, segments)
        R = _frame_from_axis(B - A)
        Vw = (V @ R.T) + 0.5 * (A + B)
        # axial coordinate in [0,1] from A to B (caps clamp)
        t = np.clip(((Vw - A) @ (B - A)) / (L * L), 0.0, 1.0)
        Vs.append(Vw)
        Fs.append(F + base)
        seg.append(np.full(len(Vw), ci, dtype=np.int32))
        skin.append(np.full(len(Vw), is_skin, dtype=np.int32))
        # LBS weights: own bone by axial fraction, blended across bone starts
        # and into the parent bone near the proximal joint.
        idx = np.zeros((len(Vw), 4), dtype=np.int32)
        w = np.zeros((len(Vw), 4), dtype=np.float64)
        starts = [b[0] for b in bones] + [1.0]
        bone_ids = [b[1] for b in bones]
        parent_bone = int(SKELETON_PARENTS[bone_ids[0]])
        if parent_bone < 0:
            parent_bone = bone_ids[0]
        for vi in range(len(Vw)):
            ti = t[vi]
            k = 0
            while k + 1 < len(bone_ids) and ti >= starts[k + 1]:
                k += 1
            own = bone_ids[k]
            slots = [(own, 1.0)]
            # blend with the next bone near its start
            if k + 1 < len(bone_ids):
                d = starts[k + 1] - ti
                if d < 0.1:
                    a = 0.5 * (1.0 - d / 0.1)
                    slots = [(own, 1.0 - a), (bone_ids[k + 1], a)]
            # blend with the previous bone (or parent) near this bone's start
            prev = bone_ids[k - 1] if k > 0 else parent_bone
            d = ti - starts[k]
            if d < 0.1 and prev != own:
                a = 0.5 * (1.0 - d / 0.1)
                slots = [(b, ww * (1.0 - a)) for b, ww in slots] + [(prev, a)]
            # fill to 4 slots (unused slots: own bone, weight 0)
            while len(slots) < 4:
                slots.append((own, 0.0))
            for s, (b, ww) in enumerate(slots[:4]):
                idx[vi, s] = b
                w[vi, s] = ww
        w /= w.sum(axis=1, keepdims=True)
        sidx.append(idx)
        sw.append(w)
        base += len(Vw)
    return dict(
        V=np.concatenate(Vs), F=np.concatenate(Fs),
        segment=np.concatenate(seg), skin=np.concatenate(skin),
        skin_idx=np.concatenate(sidx), skin_w=np.concatenate(sw),
        joints_rest=joints, parents=SKELETON_PARENTS.copy())


# ----------------------------------------------------------------------------
# Appearance and materials
# ----------------------------------------------------------------------------
def value_noise_albedo(V: np.ndarray, seed: int,
                       freqs=(2.0, 4.0, 8.0), amps=(0.5, 0.25, 0.125)) -> np.ndarray:
    """Per-vertex RGB from 3-octave value noise, rescaled to [0.1, 0.9].

    Lattice values from splitmix64; trilinear interpolation with smoothstep
    weights; octave frequencies in cycles per metre.
    """
    V = np.asarray(V, dtype=np.float64)
    out = np.zeros((len(V), 3))
    for ch in range(3):
        acc = np.zeros(len(V))
        for o, (fr, am) in enumerate(zip(freqs, amps)):
            p = V * fr
            i0 = np.floor(p)
            fr_ = p - i0
            s = fr_ * fr_ * (3.0 - 2.0 * fr_)
            i0 = i0.astype(np.int64)
            val = np.zeros(len(V))
            for dx in (0, 1):
                wx = s[:, 0] if dx else 1.0 - s[:, 0]
                for dy in (0, 1):
                    wy = s[:, 1] if dy else 1.0 - s[:, 1]
                    for dz in (0, 1):
                        wz = s[:, 2] if dz else 1.0 - s[:, 2]
                        lv = _lattice_value(i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz,
                                            seed * 97 + o * 7 + ch)
                        val += wx * wy * wz * lv
            acc += am * val
        lo, hi = acc.min(), acc.max()
        out[:, ch] = 0.1 + 0.8 * (acc - lo) / max(hi - lo, 1e-12)
    return out


def half_split_material(V: np.ndarray, seed: int, skin=1.0, cloth=0.2) -> np.ndarray:
    """Material weight 1.0 (skin) or 0.2 (cloth) by a seeded half-space."""
    rng = np.random.default_rng(seed + 1000)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    c = V.mean(axis=0)
    return np.where((V - c) @ u >= 0.0, skin, cloth)


# ----------------------------------------------------------------------------
# Rotations (FP64, for ground truth only)
# ----------------------------------------------------------------------------
def _rodrigues(aa: np.ndarray) -> np.ndarray:
    aa = np.atleast_2d(aa)
    th = np.linalg.norm(aa, axis=1)
    out = np.tile(np.eye(3), (len(aa), 1, 1))
    for i in range(len(aa)):
        if th[i] < 1e-15:
            continue
        k = aa[i] / th[i]
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        out[i] = np.eye(3) + math.sin(th[i]) * Kx + (1 - math.cos(th[i])) * (Kx @ Kx)
    return out


def _euler_xyz(a: np.ndarray) -> np.ndarray:
    """Rx(a0) Ry(a1) Rz(a2) per row (the pose convention of the skeleton)."""
    out = np.empty((len(a), 3, 3))
    for i, (x, y, z) in enumerate(a):
        cx, sx, cy, sy, cz, sz = math.cos(x), math.sin(x), math.cos(y), math.sin(y), math.cos(z), math.sin(z)
        Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
        Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
        Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
        out[i] = Rx @ Ry @ Rz
    return out


def _rbf_width(c: np.ndarray) -> float:
    n_ctrl = len(c)
    if n_ctrl < 2:
        return 0.1
    d2c = ((c[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2c, np.inf)
    return float(np.sqrt(d2c.min(axis=1)).mean())


def rbf_field(V: np.ndarray, ctrl: np.ndarray, aa: np.ndarray, tt: np.ndarray, rho: float) -> np.ndarray:
    """Blend of the control points' rigid motions (rotation ``aa`` about the
    control point, then translation ``tt``) with normalised Gaussian RBFs of
    width ``rho``: the generator's own smooth deformation model."""
    V = np.asarray(V, dtype=np.float64)
    R = _rodrigues(aa)
    out = np.empty_like(V)
    chunk = 8192
    for s in range(0, len(V), chunk):
        v = V[s:s + chunk]
        d2 = ((v[:, None, :] - ctrl[None, :, :]) ** 2).sum(-1)
        lw = -d2 / (2.0 * rho * rho)
        lw -= lw.max(axis=1, keepdims=True)
        phi = np.exp(lw)
        phi /= phi.sum(axis=1, keepdims=True)
        rel = v[:, None, :] - ctrl[None, :, :]
        moved = np.einsum("mij,nmj->nmi", R, rel) + ctrl[None] + tt[None]
        out[s:s + chunk] = np.einsum("nm,nmi->ni", phi, moved)
    return out


def smooth_deformation(V: np.ndarray, n_ctrl: int, sigma_rot: float,
                       sigma_t: float, seed: int) -> Dict[str, np.ndarray]:
    """Ground-truth non-rigid deformation on random control points.

    ``n_ctrl`` control points are a seeded random subset of the vertices; each
    gets a random rotation (axis-angle ~ N(0, sigma_rot) per axis) and
    translation (~ N(0, sigma_t)).  The field is blended with normalised
    Gaussian RBFs of width equal to the mean nearest-control-point spacing.
    Returns the deformed vertices and the draws.
    """
    rng = np.random.default_rng(seed + 2000)
    V = np.asarray(V, dtype=np.float64)
    ids = np.sort(rng.choice(len(V), size=n_ctrl, replace=False))
    c = V[ids]
    aa = rng.normal(0.0, sigma_rot, size=(n_ctrl, 3))
    tt = rng.normal(0.0, sigma_t, size=(n_ctrl, 3))
    rho = _rbf_width(c)
    return dict(V=rbf_field(V, c, aa, tt, rho), ctrl_ids=ids, aa=aa, t=tt, rho=rho)


def rbf_field_linear(V: np.ndarray, ctrl: np.ndarray, aa: np.ndarray, tt: np.ndarray, rho: float) -> np.ndarray:
    """The field of ``rbf_field`` written as one blended 3x3 matrix and
    offset per vertex (the blend of rigid motions is linear in the vertex):
    sum_m phi_m (R_m (v - c_m) + c_m + t_m) = (sum_m phi_m R_m) v
    + sum_m phi_m (c_m + t_m - R_m c_m).  Equal to ``rbf_field`` up to
    rounding and several times faster; used for long sequences."""
    V = np.asarray(V, dtype=np.float64)
    ctrl = np.asarray(ctrl, dtype=np.float64)
    R = _rodrigues(aa)
    off = ctrl + tt - np.einsum("mij,mj->mi", R, ctrl)
    out = np.empty_like(V)
    chunk = 8192
    for s in range(0, len(V), chunk):
        v = V[s:s + chunk]
        d2 = ((v[:, None, :] - ctrl[None, :, :]) ** 2).sum(-1)
        lw = -d2 / (2.0 * rho * rho)
        lw -= lw.max(axis=1, keepdims=True)
        phi = np.exp(lw)
        phi /= phi.sum(axis=1, keepdims=True)
        A = (phi @ R.reshape(-1, 9)).reshape(-1, 3, 3)
        out[s:s + chunk] = np.einsum("nij,nj->ni", A, v) + phi @ off
    return out


def ar1_draws(V: np.ndarray, n_frames: int, n_ctrl: int, sigma_rot: float, sigma_t: float,
              seed: int, rho_ar: float = 0.9):
    """Control points, RBF width and the per-frame control-point rotations
    and translations (aa, tt) of an AR(1) sequence: x_t = rho x_{t-1} +
    sqrt(1 - rho^2) sigma eps_t, started from the stationary distribution."""
    ids, rho, draws = _ar1_state(V, n_frames, n_ctrl, sigma_rot, sigma_t, seed, rho_ar)
    return np.asarray(V, dtype=np.float64)[ids], rho, draws


def _ar1_state(V, n_frames, n_ctrl, sigma_rot, sigma_t, seed, rho_ar):
    rng = np.random.default_rng(seed + 3000)
    V = np.asarray(V, dtype=np.float64)
    ids = np.sort(rng.choice(len(V), size=n_ctrl, replace=False))
    rho = _rbf_width(V[ids])
    aa = rng.normal(0.0, sigma_rot, size=(n_ctrl, 3))
    tt = rng.normal(0.0, sigma_t, size=(n_ctrl, 3))
    k = math.sqrt(1.0 - rho_ar * rho_ar)
    draws = []
    for _ in range(n_frames):
        draws.append((aa, tt))
        aa = rho_ar * aa + k * rng.normal(0.0, sigma_rot, size=aa.shape)
        tt = rho_ar * tt + k * rng.normal(0.0, sigma_t, size=tt.shape)
    return ids, rho, draws


def ar1_sequence(V: np.ndarray, n_frames: int, n_ctrl: int, sigma_rot: float, sigma_t: float,
                 seed: int, rho_ar: float = 0.9) -> List[np.ndarray]:
    """Deformed vertex positions of a sequence whose control-point rotations
    and translations follow AR(1) (``ar1_draws``)."""
    c, rho, draws = ar1_draws(V, n_frames, n_ctrl, sigma_rot, sigma_t, seed, rho_ar)
    return [rbf_field(V, c, aa, tt, rho) for aa, tt in draws]


def ar1_frame(V: np.ndarray, n_ctrl: int, sigma_rot: float, sigma_t: float, seed: int, i: int,
              rho_ar: float = 0.9) -> np.ndarray:
    """Frame i of the AR(1) sequence of ``seed`` on its own (the draws up to
    i are repeated, the field is ``rbf_field_linear``): lets a pool
    generate one long sequence's frames in parallel."""
    c, rho, draws = ar1_draws(V, i + 1, n_ctrl, sigma_rot, sigma_t, seed, rho_ar)
    aa, tt = draws[i]
    return rbf_field_linear(V, c, aa, tt, rho)


def stream_frame(scene, seed: int, i: int, n_ctrl: int = 500, sigma_pose: float = 0.1, sigma_root: float = 0.05,
                 sigma_root_t: float = 0.03, sigma_rot: float = 0.05, sigma_t: float = 0.01, rho_ar: float = 0.9,
                 noise: float = 0.01, fps: float = 25.0):
    """Frame i of a tracked stream of a body capture ``scene`` (a Scene with
    a skeleton).  Articulated motion is smooth, as a performer's: every
    joint angle and the root's rotation and translation move from the
    capture's ground-truth pose along a sinusoid, a (sin(w t + phi) -
    sin(phi)), with amplitude a ~ N(0, sigma_pose) rad per angle
    (sigma_root rad, sigma_root_t m at the root), frequency w / 2 pi
    uniform in [0.3, 1] Hz at ``fps`` frames per second and a uniform phase,
    so that frame 0 has the capture's own pose (from which its pose_init
    starts).  The posed surface is deformed by the AR(1) control-point field
    of ``ar1_draws`` (n_ctrl control points, sigma_rot rad / sigma_t m,
    rho_ar), and the frame is rendered with N(0, noise) colour noise.
    Returns (rgb, dt, mask, joints2d, joints3d) with 2 px / 1 cm detection
    noise."""
    sk, meta = scene.skeleton, scene.meta
    tpl = dict(V=np.asarray(scene.V, dtype=np.float64), joints_rest=np.asarray(sk["joints_rest"], dtype=np.float64),
               parents=sk["parents"], skin_idx=sk["skin_idx"], skin_w=sk["skin_w"])
    dof_joints = [j for j in range(1, 23) if j not in set(SKELETON_SITES.tolist())]
    rng = np.random.default_rng(seed + 7000)
    n_ang = 3 * len(dof_joints)
    amp = np.concatenate([rng.normal(0.0, sigma_pose, size=n_ang), rng.normal(0.0, sigma_root, size=3),
                          rng.normal(0.0, sigma_root_t, size=3)])
    w = 2.0 * math.pi * rng.uniform(0.3, 1.0, size=amp.size) / fps
    phi = rng.uniform(0.0, 2.0 * math.pi, size=amp.size)
    dev = amp * (np.sin(w * i + phi) - np.sin(phi))
    angles = np.zeros((23, 3))
    angles[dof_joints] = np.asarray(meta["pose_gt"][6:], dtype=np.float64).reshape(-1, 3) + dev[:n_ang].reshape(-1, 3)
    root_aa = np.asarray(meta["root_aa"], dtype=np.float64) + dev[n_ang:n_ang + 3]
    root_t = np.asarray(meta["root_t"], dtype=np.float64) + dev[n_ang + 3:]
    Vp, joints = pose_body(tpl, _rodrigues(root_aa)[0], root_t, _euler_xyz(angles))
    ids, rho, draws = _ar1_state(scene.V, i + 1, n_ctrl, sigma_rot, sigma_t, seed, rho_ar)
    aa, tt = draws[i]
    V = rbf_field_linear(Vp, Vp[ids], aa, tt, rho)
    frng = np.random.default_rng([seed, i, 11])
    rgb, dt, mask = _finish_frame(V, scene.F, scene.albedo, scene.cam, frng, noise)
    cam = scene.cam
    j3 = joints + frng.normal(0.0, 0.01, size=joints.shape)
    u = cam.f * joints[:, 0] / joints[:, 2] + cam.cx
    v = cam.f * joints[:, 1] / joints[:, 2] + cam.cy
    j2 = np.stack([u, v], 1) + frng.normal(0.0, 2.0, size=(len(joints), 2))
    return rgb, dt, mask, j2.astype(np.float32), j3.astype(np.float32)


def render_frame(V_target: np.ndarray, F: np.ndarray, albedo: np.ndarray, cam: Camera, seed: int,
                 noise: float = 0.01):
    """(rgb, dt, mask) of a target frame: rendering + N(0, noise) + the
    silhouette's contour distance transform."""
    return _finish_frame(V_target, F, albedo, cam, np.random.default_rng(seed), noise)


def pose_body(tpl: dict, root_R: np.ndarray, root_t: np.ndarray,
              local_R: np.ndarray):
    """Pose the rest body: global joint frames from local rotations, then
    linear blend skinning of the rest vertices.  Returns (V_posed, joints)."""
    J = tpl["joints_rest"]
    par = tpl["parents"]
    n = len(par)
    G = np.zeros((n, 3, 3))
    o = np.zeros((n, 3))
    for j in range(n):
        if par[j] < 0:
            G[j] = root_R
            o[j] = root_t
        else:
            p = par[j]
            o[j] = o[p] + G[p] @ (J[j] - J[p])
            G[j] = G[p] @ local_R[j]
    V = tpl["V"]
    out = np.zeros_like(V)
    for s in range(4):
        b = tpl["skin_idx"][:, s]
        w = tpl["skin_w"][:, s]
        moved = np.einsum("nij,nj->ni", G[b], V - J[b]) + o[b]
        out += w[:, None] * moved
    return out, o


# ----------------------------------------------------------------------------
# Rendering (FP64 floating-point coverage, perspective-correct colours)
# ----------------------------------------------------------------------------
def render(Vw: np.ndarray, F: np.ndarray, colors: np.ndarray, cam: Camera):
    """Z-buffered rendering of a coloured mesh at pixel centres.

    Coverage uses FP64 barycentrics (closed triangles); colours are
    interpolated perspective-correctly.  Background is black.
    Returns (rgb (H,W,3) float64, mask (H,W) bool).
    """
    Vw = np.asarray(Vw, dtype=np.float64)
    X, Y, Z = Vw[:, 0], Vw[:, 1], Vw[:, 2]
    ok = Z > 1e-3
    Zs = np.where(ok, Z, 1.0)
    u = cam.f * X / Zs + cam.cx
    v = cam.f * Y / Zs + cam.cy
    F = np.asarray(F, dtype=np.int64)
    tri_ok = ok[F].all(axis=1)
    Ft = F[tri_ok]
    tu, tv, tz = u[Ft], v[Ft], Z[Ft]
    x0 = np.clip(np.ceil(tu.min(1)), 0, cam.W - 1).astype(np.int64)
    x1 = np.clip(np.floor(tu.max(1)), -1, cam.W - 1).astype(np.int64)
    y0 = np.clip(np.ceil(tv.min(1)), 0, cam.H - 1).astype(np.int64)
    y1 = np.clip(np.floor(tv.max(1)), -1, cam.H - 1).astype(np.int64)
    bw = x1 - x0 + 1
    bh = y1 - y0 + 1
    keep = (bw > 0) & (bh > 0) & (tu.max(1) >= 0) & (tv.max(1) >= 0) \
        & (tu.min(1) <= cam.W - 1) & (tv.min(1) <= cam.H - 1)
    idx = np.nonzero(keep)[0]
    order = idx[np.lexsort((bh[idx], bw[idx]))]
    pix_all, z_all, col_all = [], [], []
    chunk = 2048
    for s in range(0, len(order), chunk):
        ids = order[s:s + chunk]
        mw, mh = int(bw[ids].max()), int(bh[ids].max())
        gx = x0[ids, None, None] + np.arange(mw)[None, None, :]
        gy = y0[ids, None, None] + np.arange(mh)[None, :, None]
        gx = np.broadcast_to(gx, (len(ids), mh, mw))
        gy = np.broadcast_to(gy, (len(ids), mh, mw))
        inb = (gx <= x1[ids, None, None]) & (gy <= y1[ids, None, None])
        ax, ay = tu[ids, 0, None, None], tv[ids, 0, None, None]
        bx, by = tu[ids, 1, None, None], tv[ids, 1, None, None]
        cx, cy = tu[ids, 2, None, None], tv[ids, 2, None, None]
        area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
        w0 = (bx - gx) * (cy - gy) - (by - gy) * (cx - gx)
        w1 = (cx - gx) * (ay - gy) - (cy - gy) * (ax - gx)
        w2 = (ax - gx) * (by - gy) - (ay - gy) * (bx - gx)
        nz = np.abs(area) > 1e-18
        sa = np.where(nz, area, 1.0)
        b0, b1, b2 = w0 / sa, w1 / sa, w2 / sa
        inside = inb & nz & (b0 >= 0) & (b1 >= 0) & (b2 >= 0)
        zi = tz[ids]
        invz = b0 / zi[:, 0, None, None] + b1 / zi[:, 1, None, None] + b2 / zi[:, 2, None, None]
        depth = 1.0 / np.where(inside, invz, 1.0)
        cc = colors[Ft[ids]]  # (n,3 verts,3 ch)
        col = (b0[..., None] * cc[:, None, None, 0, :] / zi[:, 0, None, None, None]
               + b1[..., None] * cc[:, None, None, 1, :] / zi[:, 1, None, None, None]
               + b2[..., None] * cc[:, None, None, 2, :] / zi[:, 2, None, None, None]) \
            * depth[..., None]
        m = inside
        pix_all.append((gy[m] * cam.W + gx[m]))
        z_all.append(depth[m])
        col_all.append(col[m])
    rgb = np.zeros((cam.H * cam.W, 3))
    mask = np.zeros(cam.H * cam.W, dtype=bool)
    if pix_all:
        pix = np.concatenate(pix_all)
        if len(pix):
            z = np.concatenate(z_all)
            col = np.concatenate(col_all)
            o = np.lexsort((z, pix))
            pix_s = pix[o]
            first = np.ones(len(pix_s), dtype=bool)
            first[1:] = pix_s[1:] != pix_s[:-1]
            sel = o[first]
            rgb[pix[sel]] = col[sel]
            mask[pix[sel]] = True
    return rgb.reshape(cam.H, cam.W, 3), mask.reshape(cam.H, cam.W)


def contour_distance_transform(mask: np.ndarray) -> np.ndarray:
    """Euclidean distance (pixels) from each pixel centre to the nearest
    contour pixel: a foreground pixel with a 4-neighbour in the background or
    on the image border.  Zero on contour pixels.  An empty mask gives zeros.
    """
    m = np.asarray(mask, dtype=bool)
    pad = np.pad(m, 1, constant_values=False)
    interior = pad[1:-1, 1:-1] & pad[:-2, 1:-1] & pad[2:, 1:-1] & pad[1:-1, :-2] & pad[1:-1, 2:]
    contour = m & ~interior
    if not contour.any():
        return np.zeros(m.shape, dtype=np.float64)
    return ndimage.distance_transform_edt(~contour)


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------
# Weights of the per-vertex surface stage.  The paper's values (w_photo 1e4,
# w_silhouette 600, w_smooth 10, w_edge 30, w_velocity 0.25, w_acceleration
# 0.1) read with positions in millimetres; the regularisers are rescaled by
# 1e6 for metres and all weights by 1e-4 so that w_photo = 1 as in the graph
# stage, whose silhouette weight 0.1 is kept.
SURFACE_WEIGHTS = (1.0, 0.1, 1.0e3, 3.0e3, 25.0, 10.0)


@dataclasses.dataclass
class Scene:
    """Everything one capture needs, as FP32/int32 arrays ready for upload."""

    name: str
    cam: Camera
    V: np.ndarray          # (N,3) f32 rest template
    F: np.ndarray          # (T,3) i32
    albedo: np.ndarray     # (N,3) f32
    material: np.ndarray   # (N,) f32
    rgb: np.ndarray        # (H,W,3) f32 target frame
    dt: np.ndarray         # (H,W) f32 silhouette distance transform
    mask: np.ndarray       # (H,W) bool
    n_nodes: int
    K: int
    n_gn: int
    n_pcg: int
    weights: tuple         # (w_photo, w_sil, w_arap)
    V_gt: np.ndarray       # (N,3) f64 ground-truth surface
    skeleton: Optional[dict] = None   # body scenes only
    joints2d: Optional[np.ndarray] = None
    joints3d: Optional[np.ndarray] = None
    pose_init: Optional[np.ndarray] = None   # (57,) f32
    n_gn_pose: int = 5
    # per-vertex surface stage: (w_photo, w_sil, w_smooth, w_edge, w_velocity,
    # w_acceleration) and its Gauss-Newton / PCG counts
    surface_weights: tuple = SURFACE_WEIGHTS
    n_gn_surface: int = 3
    n_pcg_surface: int = 4
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.V)


def _finish_frame(V_target, F, albedo, cam, rng, noise=0.01):
    rgb, mask = render(V_target, F, albedo, cam)
    rgb = rgb + rng.normal(0.0, noise, size=rgb.shape)
    dt = contour_distance_transform(mask)
    return rgb.astype(np.float32), dt.astype(np.float32), mask


def make_scene(name: str, seed: Optional[int] = None, **over) -> Scene:
    """Build one seeded capture.

    ``tiny``   capsule (1,002 v / 2,000 t), 64 nodes K=4, 128^2, f=150,
               GT rotations sigma 0.05 rad, translations 0.01 m, 5 GN x 20 PCG.
    ``body``   articulated body (6,020 v / 12,000 t), 500 nodes K=4, 1024^2,
               f=1200, GT pose + non-rigid rotations sigma 0.1 rad,
               2D joints with 2 px noise, 3D joints with 1 cm noise,
               10 GN x 40 PCG after a 5-step pose fit.
    ``stress`` body of ~100k vertices, 4,000 nodes, K=8, 2048^2, f=2400.
    Keyword overrides: rings, segments, n_nodes, K, side, n_gn, n_pcg; frame=False
    (body and stress) skips the target frame (rgb, dt and mask are None).
    """
    if name == "tiny":
        seed = 0 if seed is None else seed
        rng = np.random.default_rng(seed)
        V, F = capsule_mesh(0.3, 1.0, over.get("rings", 40), over.get("segments", 25))
        V = V + np.array([0.0, 0.0, 3.0])
        side = over.get("side", 128)
        cam = Camera(f=150.0 * side / 128.0, W=side, H=side)
        V32 = V.astype(np.float32)
        albedo = value_noise_albedo(V32.astype(np.float64), seed)
        material = half_split_material(V32.astype(np.float64), seed)
        n_nodes = over.get("n_nodes", 64)
        gt = smooth_deformation(V32.astype(np.float64), n_nodes, 0.05, 0.01, seed)
        rgb, dt, mask = _finish_frame(gt["V"], F, albedo, cam, rng)
        return Scene("tiny", cam, V32, F.astype(np.int32), albedo.astype(np.float32),
                     material.astype(np.float32), rgb, dt, mask, n_nodes,
                     over.get("K", 4), over.get("n_gn", 5), over.get("n_pcg", 20),
                     (1.0, 0.1, 10.0), gt["V"], meta=dict(seed=seed))
    if name in ("body", "stress"):
        stress = name == "stress"
        seed = (1 if not stress else 4) if seed is None else seed
        rng = np.random.default_rng(seed)
        rings = over.get("rings", 24 if not stress else 100)
        segs = over.get("segments", 25 if not stress else 100)
        tpl = body_template(rings, segs)
        V = tpl["V"]
        F = tpl["F"]
        side = over.get("side", 1024 if not stress else 2048)
        cam = Camera(f=1200.0 * side / 1024.0, W=side, H=side)
        V32 = V.astype(np.float32)
        albedo = value_noise_albedo(V32.astype(np.float64), seed)
        material = np.where(tpl["skin"] > 0, 1.0, 0.2)
        n_nodes = over.get("n_nodes", 500 if not stress else 4000)
        # ground-truth pose: small global rotation, Euler XYZ joint angles
        # ~N(0, 0.2); the frame starts from the ground truth perturbed by
        # N(0, 0.05) rad per angle and N(0, 2 cm) at the root, like a pose
        # extrapolated from the previous two frames
        root_aa = rng.normal(0.0, 0.05, size=3)
        root_t = tpl["joints_rest"][0] + rng.normal(0.0, 0.03, size=3)
        angles = rng.normal(0.0, over.get("sigma_pose", 0.2), size=(23, 3))
        angles[SKELETON_SITES] = 0.0
        angles[0] = 0.0
        local = _euler_xyz(angles)
        Vp, joints_gt = pose_body(dict(tpl, V=V32.astype(np.float64)),
                                  _rodrigues(root_aa)[0], root_t, local)
        if over.get("frame", True):
            gt = smooth_deformation(Vp, n_nodes, over.get("sigma_nonrigid", 0.1), 0.01, seed)
            rgb, dt, mask = _finish_frame(gt["V"], F, albedo, cam, rng)
        else:
            # no target frame (streams render their own): the generator's
            # draws stay those of the full scene
            gt = dict(V=Vp)
            rgb = dt = mask = None
            rng.normal(0.0, 0.01, size=(side, side, 3))
        j3 = joints_gt + rng.normal(0.0, 0.01, size=joints_gt.shape)
        u = cam.f * joints_gt[:, 0] / joints_gt[:, 2] + cam.cx
        v = cam.f * joints_gt[:, 1] / joints_gt[:, 2] + cam.cy
        j2 = np.stack([u, v], 1) + rng.normal(0.0, 2.0, size=(23, 2))
        dof_joints = [j for j in range(1, 23) if j not in set(SKELETON_SITES.tolist())]
        pose_gt = np.concatenate([root_aa, root_t] + [angles[j] for j in dof_joints])
        pose0 = pose_gt.copy()
        pose0[:3] += rng.normal(0.0, 0.02, size=3)
        pose0[3:6] += rng.normal(0.0, 0.02, size=3)
        pose0[6:] += rng.normal(0.0, over.get("sigma_init", 0.05), size=len(pose0) - 6)
        skel = dict(parents=tpl["parents"], joints_rest=tpl["joints_rest"].astype(np.float32),
                    skin_idx=tpl["skin_idx"].astype(np.int32),
                    skin_w=tpl["skin_w"].astype(np.float32),
                    segment=tpl["segment"], bone_part=SKELETON_BONE_PART.copy(), torso_part=TORSO_PART)
        return Scene(name, cam, V32, F.astype(np.int32), albedo.astype(np.float32),
                     material.astype(np.float32), rgb, dt, mask, n_nodes,
                     over.get("K", 4 if not stress else 8),
                     over.get("n_gn", 10), over.get("n_pcg", 40), (1.0, 0.1, 10.0),
                     gt["V"], skeleton=skel, joints2d=j2.astype(np.float32),
                     joints3d=j3.astype(np.float32), pose_init=pose0.astype(np.float32),
                     meta=dict(seed=seed, root_aa=root_aa, root_t=root_t, pose_gt=pose_gt,
                               joints_gt=joints_gt, V_posed=Vp))
    raise ValueError(f"unknown scene {name!r}")


def batch_specs(count: int = 64, seed: int = 2, n_min=2000, n_max=20000, side_min=256, side_max=1024):
    """Per-capture (scene seed, rings, image side, nodes) of an uneven batch:
    vertices log-uniform in [n_min, n_max] (articulated capsule bodies with a
    variable ring count), nodes = vertices / 12, square images log-uniform in
    [side_min, side_max] rounded to a multiple of 32."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        n_target = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        rings = max(4, int(round((n_target / 10.0 - 2.0) / 25.0)))
        side = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max))) / 32.0)) * 32
        n_vert = 10 * (2 + rings * 25)
        out.append((1000 + seed * 100 + c, rings, side, max(8, n_vert // 12)))
    return out


def make_batch_member(spec) -> Scene:
    scene_seed, rings, side, n_nodes = spec
    return make_scene("body", seed=scene_seed, rings=rings, segments=25, side=side, n_nodes=n_nodes)


def make_batch(count: int = 64, seed: int = 2, n_min=2000, n_max=20000,
               side_min=256, side_max=1024) -> List[Scene]:
    """Uneven captures (``batch_specs``), generated one after the other."""
    return [make_batch_member(sp) for sp in batch_specs(count, seed, n_min, n_max, side_min, side_max)]
