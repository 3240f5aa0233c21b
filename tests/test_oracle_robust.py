"""Pins for the robust colour kernel sigma_c of E_photo (Sec. 3.4) in the
oracle (oracle.nonrigid.prune, used by the graph and the surface stage):
off and huge thresholds change nothing, a tiny one drops every photometric
row, the kept set is exactly {||I(pi(v)) - C|| <= sigma_c}, and the
Jacobian of the remaining rows matches finite differences with the
decisions frozen."""
import copy

import numpy as np

import synth
from oracle import graph as ograph
from oracle import nonrigid as nr
from oracle import surface as sf


def _problem():
    scene = synth.make_scene("tiny")
    g = ograph.build_graph(scene.V, scene.material, scene.n_nodes, scene.K)
    P = nr.problem_from_scene(scene, g)
    R, t = nr.identity_params(P.n)
    nr.frame_decisions(P, scene.F, R, t)
    return scene, P, R, t


def test_thresholds_off_huge_tiny():
    scene, P, R, t = _problem()
    F0, J0 = nr.linearise(P, R, t)
    Q = copy.copy(P)
    Q.sigma_c = 1e9
    F1, J1 = nr.linearise(Q, R, t)
    assert np.array_equal(F0, F1) and (J0 != J1).nnz == 0
    Q.sigma_c = 1e-9
    vr = nr.vertex_residuals(Q, R, t)
    assert not vr["photo_on"].any() and (vr["photo"] == 0).all()
    assert vr["sil_on"].sum() == nr.vertex_residuals(P, R, t)["sil_on"].sum()


def test_kept_set_is_the_colour_ball():
    scene, P, R, t = _problem()
    vr0 = nr.vertex_residuals(P, R, t)
    d = np.linalg.norm(vr0["photo"], axis=1) / np.sqrt(P.w_photo)     # ||I - C|| of the active ones
    sigma = float(np.median(d[vr0["photo_on"]]))
    Q = copy.copy(P)
    Q.sigma_c = sigma
    vr = nr.vertex_residuals(Q, R, t)
    assert np.array_equal(vr["photo_on"], vr0["photo_on"] & (d <= sigma))
    kept = vr["photo_on"].sum()
    assert 0.3 * vr0["photo_on"].sum() < kept < 0.7 * vr0["photo_on"].sum()
    e = nr.energy(Q, R, t)
    assert np.isclose(e["photo"], float((vr0["photo"][vr["photo_on"]] ** 2).sum()), rtol=1e-12)
    # the surface stage prunes the same way
    S = sf.problem_from_scene(scene)
    S.vis, S.inB, S.bsign = P.vis, P.inB, P.bsign
    S.sigma_c = sigma
    rs = sf.residuals(S, S.base)
    assert np.array_equal(rs["photo_on"], vr["photo_on"])


def _affine(P):
    """Per-channel affine images: bilinear sampling and central differences
    are exact there, so the assembled J must equal finite differences."""
    Q = copy.copy(P)
    yy, xx = np.mgrid[:P.H, :P.W].astype(np.float64)
    Q.rgb = np.stack([0.5 + 0.004 * xx - 0.002 * yy, 0.3 - 0.003 * xx + 0.005 * yy,
                      0.4 + 0.001 * xx + 0.001 * yy], axis=-1)
    Q.dt = 2.0 + 0.05 * xx + 0.03 * yy
    Q._grad_rgb = None
    Q._grad_dt = None
    return Q


def test_jacobian_fd_with_frozen_decisions():
    scene, P, R, t = _problem()
    P = _affine(P)
    rng = np.random.default_rng(2)
    R = nr.so3_exp(rng.normal(scale=0.03, size=(P.n, 3))) @ R
    t = t + rng.normal(scale=0.003, size=t.shape)
    Q = copy.copy(P)
    Q.tris = None
    vr0 = nr.vertex_residuals(Q, R, t)
    d = np.linalg.norm(vr0["photo"], axis=1) / np.sqrt(P.w_photo)
    Q.sigma_c = float(np.median(d[vr0["photo_on"]]))
    Q.pruned = vr0["photo_on"] & (d > Q.sigma_c)
    F, J = nr.linearise(Q, R, t)
    vr = nr.vertex_residuals(Q, R, t)
    assert not (vr["photo_on"] & Q.pruned).any()
    # silhouette rows of J carry the direction sign b_i (Sec. 3.4)
    n_p = 3 * int(vr["photo_on"].sum())
    on_s = vr["sil_on"]
    sgn = np.ones(len(F))
    sgn[n_p:n_p + int(on_s.sum())] = Q.bsign[on_s]
    h = 1e-6
    cols = rng.choice(6 * P.n, 40, replace=False)
    for c in cols:
        dp = np.zeros(6 * P.n)
        dp[c] = h
        Rp, tp = nr.apply_update(R, t, dp)
        Rm, tm = nr.apply_update(R, t, -dp)
        Fp, _ = nr.linearise(Q, Rp, tp)
        Fm, _ = nr.linearise(Q, Rm, tm)
        fd = sgn * (Fp - Fm) / (2 * h)
        col = J.tocsc()[:, c].toarray().ravel()
        assert np.abs(fd - col).max() <= 1e-6 * max(1.0, np.abs(col).max()), c
