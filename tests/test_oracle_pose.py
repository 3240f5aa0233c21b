"""Pins for the pose-stage oracle (CPU).

* Euler convention vs SciPy's intrinsic XYZ rotations.
* Rest pose skins to the template; a global root motion moves every joint
  and vertex rigidly (closed form).
* Finite-difference Jacobian with an affine distance-transform stand-in
  (bilinear sampling and central differences exact), b_i signs folded in.
* Cholesky solve vs numpy.linalg.solve; a non-positive pivot raises.
* Noise-free detections generated at a known pose are recovered.
* E_temporal and E_anatomic: their Jacobian rows by finite differences; the
  barrier's energy and Gauss-Newton step against closed forms; E_temporal
  alone pulls the joints onto a reachable previous frame's joints.
* The frame-start extrapolation is exact for constant-velocity motion.
"""
import copy

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from oracle import nonrigid as nr
from oracle import pose as op


@pytest.fixture(scope="module")
def body():
    return synth.make_scene("body")


def test_euler_matches_scipy():
    a = np.random.default_rng(0).normal(scale=0.7, size=(20, 3))
    ref = Rotation.from_euler("XYZ", a).as_matrix()
    assert np.abs(op.euler_xyz(a) - ref).max() < 1e-14


def test_rest_pose_and_rigid_root(body):
    pb = op.problem_from_scene(body)
    sk = pb.sk
    rest = np.zeros(sk.n_dof)
    rest[3:6] = sk.joints_rest[0]
    R, t, ang = op.split_pose(sk, rest)
    G, o = op.forward_kinematics(sk, R, t, ang)
    _, VS = op.skin(sk, pb.V, G, o)
    # the skinning weights are FP32: sum_s w_is = 1 only to within rounding
    wtol = 2.0 * np.abs(sk.skin_w.sum(1) - 1.0).max() * np.abs(pb.V).max() + 1e-13
    assert np.abs(o - sk.joints_rest).max() < 1e-15
    assert np.abs(VS - pb.V).max() <= wtol
    Rg = nr.so3_exp(np.array([0.2, -0.3, 0.1]))[0]
    tg = np.array([0.05, -0.02, 0.1])
    moved = rest.copy()
    moved[:3] = nr.so3_log(Rg)[0]
    moved[3:6] = Rg @ sk.joints_rest[0] + tg
    R, t, ang = op.split_pose(sk, moved)
    G, o = op.forward_kinematics(sk, R, t, ang)
    _, VS2 = op.skin(sk, pb.V, G, o)
    assert np.abs(o - (sk.joints_rest @ Rg.T + tg)).max() < 1e-12
    assert np.abs(VS2 - (pb.V @ Rg.T + tg)).max() <= wtol + 1e-12


def _affine_dt(pb):
    Q = copy.copy(pb)
    yy, xx = np.mgrid[:pb.H, :pb.W].astype(np.float64)
    Q.dt = 3.0 + 0.02 * xx - 0.015 * yy
    Q._gdt = None
    return Q


def test_jacobian_fd(body):
    pb = _affine_dt(op.problem_from_scene(body))
    pose0 = np.asarray(body.pose_init, dtype=np.float64)
    op.frame_decisions(op.problem_from_scene(body), pose0)
    dec = op.problem_from_scene(body)
    op.frame_decisions(dec, pose0)
    pb.inB, pb.bsign = dec.inB, dec.bsign
    rng = np.random.default_rng(3)
    pose = pose0.copy()
    pose[6:] += rng.normal(scale=0.05, size=len(pose) - 6)
    F, J = op.residuals_and_jacobian(pb, pose)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for d in range(J.shape[1]):
        e = np.zeros(J.shape[1])
        e[d] = h
        Fp, _ = op.residuals_and_jacobian(pb, op.apply_update(pb.sk, pose, e))
        Fm, _ = op.residuals_and_jacobian(pb, op.apply_update(pb.sk, pose, -e))
        assert len(Fp) == len(F) == len(Fm)
        Jfd[:, d] = (Fp - Fm) / (2 * h)
    # silhouette rows carry b_i
    R, t, ang = op.split_pose(pb.sk, pose)
    G, o = op.forward_kinematics(pb.sk, R, t, ang)
    _, VS = op.skin(pb.sk, pb.V, G, o)
    _, _, _, okj, _ = op._proj(pb, o)
    _, _, _, _, inimg = op._proj(pb, VS)
    sel = np.nonzero(pb.inB & inimg)[0]
    r0 = 2 * int(okj.sum()) + 3 * len(o)
    Jfd[r0:r0 + len(sel)] *= pb.bsign[sel][:, None]
    assert len(sel) > 50
    err = np.abs(J - Jfd).max() / np.abs(Jfd).max()
    assert err < 1e-6, err


def test_cholesky():
    rng = np.random.default_rng(1)
    M = rng.normal(size=(57, 57))
    A = M @ M.T + 57 * np.eye(57)
    b = rng.normal(size=57)
    assert np.allclose(op.cholesky_solve(A, b), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        op.cholesky_solve(-np.eye(3), np.ones(3))


def test_noise_free_recovery(body):
    pb = op.problem_from_scene(body, lam_prior=1e-6)
    pb.lam_sil = 0.0
    # 3D residuals weighted as if in millimetres: with metres the 3D term is
    # too weak to rule out depth-flipped limb poses that match the 2D joints
    pb.lam_3d = 28.0e6
    gt = body.meta["pose_gt"]
    R, t, ang = op.split_pose(pb.sk, gt)
    G, o = op.forward_kinematics(pb.sk, R, t, ang)
    pb.j3d = o.copy()
    pb.j2d = np.stack([pb.f * o[:, 0] / o[:, 2] + pb.cx, pb.f * o[:, 1] / o[:, 2] + pb.cy], 1)
    pose, hist = op.gauss_newton(pb, np.asarray(body.pose_init, dtype=np.float64), 25)
    R, t, ang = op.split_pose(pb.sk, pose)
    G2, o2 = op.forward_kinematics(pb.sk, R, t, ang)
    assert np.abs(o2 - o).max() < 1e-6
    assert hist[-1]["energy"] < 1e-9 * hist[0]["energy"]


def test_pose_stage_improves_joints(body):
    out = op.solve_scene(body)
    pb = out["problem"]
    R, t, ang = op.split_pose(pb.sk, np.asarray(body.pose_init, dtype=np.float64))
    _, o0 = op.forward_kinematics(pb.sk, R, t, ang)
    e_init = np.linalg.norm(o0 - body.meta["joints_gt"], axis=1).mean()
    e_fin = np.linalg.norm(out["joints"] - body.meta["joints_gt"], axis=1).mean()
    assert out["e1"] < out["e0"]
    assert e_fin < 1.5 * e_init


def _terms_problem(body, pose):
    """A problem with E_temporal and E_anatomic switched on around `pose`:
    previous joints a few cm away, limits that leave some DOFs outside."""
    pb = op.problem_from_scene(body)
    rng = np.random.default_rng(11)
    R, t, ang = op.split_pose(pb.sk, pose)
    _, o = op.forward_kinematics(pb.sk, R, t, ang)
    pb.prev_joints = o + rng.normal(scale=0.02, size=o.shape)
    pb.temporal_w = rng.uniform(1.0, 2.5, size=len(o))
    lo = np.full(pb.sk.n_dof, -np.inf)
    hi = np.full(pb.sk.n_dof, np.inf)
    lo[6:] = pose[6:] - rng.uniform(-0.05, 0.3, size=pb.sk.n_dof - 6)
    hi[6:] = pose[6:] + rng.uniform(-0.05, 0.3, size=pb.sk.n_dof - 6)
    lo[6:], hi[6:] = np.minimum(lo[6:], hi[6:] - 0.01), np.maximum(hi[6:], lo[6:] + 0.01)
    pb.theta_min, pb.theta_max = lo, hi
    return pb


def test_temporal_and_anatomic_jacobian_fd(body):
    pose = np.asarray(body.pose_init, dtype=np.float64).copy()
    pb = _affine_dt(_terms_problem(body, pose))
    dec = op.problem_from_scene(body)
    op.frame_decisions(dec, pose)
    pb.inB, pb.bsign = dec.inB, dec.bsign
    n_active = int(((pose[6:] > pb.theta_max[6:]) | (pose[6:] < pb.theta_min[6:])).sum())
    assert n_active >= 3
    # stay clear of the limits by more than the FD step
    margin = np.minimum(np.abs(pose[6:] - pb.theta_max[6:]), np.abs(pose[6:] - pb.theta_min[6:]))
    assert margin.min() > 1e-4
    F, J = op.residuals_and_jacobian(pb, pose)
    Jn = len(pb.sk.parents)
    r_t = len(F) - (pb.sk.n_dof - 6) - n_active - 3 * Jn     # first temporal row
    h = 1e-6
    for d in range(J.shape[1]):
        e = np.zeros(J.shape[1])
        e[d] = h
        Fp, _ = op.residuals_and_jacobian(pb, op.apply_update(pb.sk, pose, e))
        Fm, _ = op.residuals_and_jacobian(pb, op.apply_update(pb.sk, pose, -e))
        fd = (Fp - Fm) / (2 * h)
        rows = slice(r_t, len(F))
        assert np.abs(fd[rows] - J[rows, d]).max() <= 1e-6 * max(1.0, np.abs(J[rows]).max()), d


def test_anatomic_barrier_closed_form(body):
    pose = np.asarray(body.pose_init, dtype=np.float64).copy()
    pb = _terms_problem(body, pose)
    pb.prev_joints = None
    pb.lam_2d = pb.lam_3d = pb.lam_sil = 0.0
    lam_a, lam_p = pb.lam_anatomic, pb.lam_prior
    th, lo, hi = pose[6:], pb.theta_min[6:], pb.theta_max[6:]
    psi = np.where(th > hi, (th - hi) ** 2, np.where(th < lo, (lo - th) ** 2, 0.0))
    assert op.energy(pb, pose) == pytest.approx(lam_a * psi.sum(), rel=1e-12)
    # prior + barrier only: the Euler block of the normal equations is
    # diagonal, and its Gauss-Newton step from the prior's centre lands on the
    # quadratic minimiser (lam_p th0 + lam_a bound) / (lam_p + lam_a)
    F, J = op.residuals_and_jacobian(pb, pose)
    A = J.T @ J
    g = -(J.T @ F)
    Ae = A[6:, 6:]
    assert np.abs(Ae - np.diag(np.diag(Ae))).max() == 0.0
    active = (th > hi) | (th < lo)
    assert np.allclose(np.diag(Ae), lam_p + lam_a * active, rtol=1e-14)
    bound = np.where(th > hi, hi, np.where(th < lo, lo, th))
    expect = np.where(active, (lam_p * th + lam_a * bound) / (lam_p + lam_a), th)
    assert np.abs(th + g[6:] / np.diag(Ae) - expect).max() < 1e-12
    # inside the limits the term is zero
    pb.theta_min[6:] = th - 1.0
    pb.theta_max[6:] = th + 1.0
    assert op.energy(pb, pose) == 0.0


def test_temporal_term_recovers_previous_joints(body):
    """Only E_temporal (with a weak prior): Gauss-Newton moves the joints onto
    the previous frame's joints when those come from a reachable pose."""
    pb = op.problem_from_scene(body, lam_prior=1e-6)
    pb.lam_2d = pb.lam_3d = pb.lam_sil = 0.0
    pb.lam_temporal = 1.0e6
    gt = body.meta["pose_gt"]
    R, t, ang = op.split_pose(pb.sk, gt)
    _, o = op.forward_kinematics(pb.sk, R, t, ang)
    pb.prev_joints = o
    pose, hist = op.gauss_newton(pb, np.asarray(body.pose_init, dtype=np.float64), 25)
    R, t, ang = op.split_pose(pb.sk, pose)
    _, o2 = op.forward_kinematics(pb.sk, R, t, ang)
    assert np.abs(o2 - o).max() < 1e-6


def test_extrapolation_is_exact_for_constant_velocity():
    rng = np.random.default_rng(12)
    n = 57
    p0 = rng.normal(scale=0.3, size=n)
    v = rng.normal(scale=0.05, size=n)
    w = rng.normal(scale=0.1, size=3)
    R0 = nr.so3_exp(p0[None, :3])[0]
    poses = []
    for k in range(3):
        p = p0 + k * v
        p[:3] = nr.so3_log(nr.so3_exp(k * w[None])[0] @ R0)[0]
        poses.append(p)
    ext = op.extrapolate(poses[1], poses[0])
    assert np.abs(ext[3:] - poses[2][3:]).max() < 1e-12
    assert np.abs(nr.so3_exp(ext[None, :3])[0] - nr.so3_exp(poses[2][None, :3])[0]).max() < 1e-12
    assert np.array_equal(op.extrapolate(poses[1]), poses[1])


def test_skinned_displacement_special_cases(body):
    """d^S = dhat at the rest pose; a pure root rotation R rotates every
    displacement by R (every bone carries R, so does their blend)."""
    pb = op.problem_from_scene(body)
    sk = pb.sk
    rng = np.random.default_rng(11)
    dhat = rng.normal(scale=0.01, size=(len(pb.V), 3))
    rest = np.zeros(sk.n_dof)
    rest[3:6] = body.skeleton["joints_rest"][0]
    assert np.abs(op.skinned_displacement(sk, rest, dhat) - dhat).max() <= 1e-15
    rot = rest.copy()
    rot[:3] = [0.3, -0.2, 0.5]
    R = nr.so3_exp(rot[:3][None])[0]
    assert np.abs(op.skinned_displacement(sk, rot, dhat) - dhat @ R.T).max() <= 1e-14


def test_jacobian_fd_with_displacement(body):
    """The displacement is held fixed: the silhouette rows of the displaced
    model still match finite differences, and a zero displacement changes
    nothing."""
    pose0 = np.asarray(body.pose_init, dtype=np.float64)
    base = op.problem_from_scene(body)
    op.frame_decisions(base, pose0)
    F0, J0 = op.residuals_and_jacobian(base, pose0)
    z = op.problem_from_scene(body)
    z.disp = np.zeros((len(z.V), 3))
    op.frame_decisions(z, pose0)
    Fz, Jz = op.residuals_and_jacobian(z, pose0)
    assert np.array_equal(F0, Fz) and np.array_equal(J0, Jz)
    rng = np.random.default_rng(12)
    dhat = 0.004 * np.sin(base.V @ rng.normal(size=(3, 3)) * 5.0)
    dec = op.problem_from_scene(body)
    dec.disp = op.skinned_displacement(dec.sk, pose0, dhat)
    op.frame_decisions(dec, pose0)
    assert (dec.inB != base.inB).any()          # the displaced model has its own contour set
    pb = _affine_dt(dec)
    pb.inB, pb.bsign, pb.disp = dec.inB, dec.bsign, dec.disp
    pose = pose0.copy()
    pose[6:] += rng.normal(scale=0.05, size=len(pose) - 6)
    F, J = op.residuals_and_jacobian(pb, pose)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for d in range(J.shape[1]):
        e = np.zeros(J.shape[1])
        e[d] = h
        Fp, _ = op.residuals_and_jacobian(pb, op.apply_update(pb.sk, pose, e))
        Fm, _ = op.residuals_and_jacobian(pb, op.apply_update(pb.sk, pose, -e))
        assert len(Fp) == len(F) == len(Fm)
        Jfd[:, d] = (Fp - Fm) / (2 * h)
    R, t, ang = op.split_pose(pb.sk, pose)
    G, o = op.forward_kinematics(pb.sk, R, t, ang)
    _, VS = op.skin(pb.sk, pb.V, G, o)
    _, _, _, okj, _ = op._proj(pb, o)
    _, _, _, _, inimg = op._proj(pb, VS + pb.disp)
    sel = np.nonzero(pb.inB & inimg)[0]
    r0 = 2 * int(okj.sum()) + 3 * len(o)
    Jfd[r0:r0 + len(sel)] *= pb.bsign[sel][:, None]
    err = np.abs(J - Jfd).max() / np.abs(Jfd).max()
    assert err < 1e-6, err
