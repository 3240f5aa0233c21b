"""Pins for the oracle's warp, rotations, sampling and ARAP (CPU)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import nonrigid as nr


def test_so3_exp_matches_scipy():
    w = np.random.default_rng(0).normal(scale=0.8, size=(50, 3))
    w[0] = 0.0
    w[1] = 1e-10
    ref = Rotation.from_rotvec(w).as_matrix()
    assert np.abs(nr.so3_exp(w) - ref).max() < 1e-14
    assert np.allclose(nr.so3_log(nr.so3_exp(w)), w, atol=1e-12)


def test_hat_is_cross_product():
    a, b = np.random.default_rng(1).normal(size=(2, 3))
    assert np.allclose(nr.hat(a) @ b, np.cross(a, b))


def test_identity_reproduces_template(tiny_problem):
    P = tiny_problem
    R, t = nr.identity_params(P.n)
    assert np.array_equal(nr.warp(P, R, t), P.base)


def _global_rigid(P, seed):
    rng = np.random.default_rng(seed)
    Rg = nr.so3_exp(rng.normal(scale=0.3, size=3))[0]
    tg = rng.normal(scale=0.1, size=3)
    R = np.tile(Rg, (P.n, 1, 1))
    t = (P.g @ Rg.T) + tg - P.g           # R_k = R, t_k = R g_k + t - g_k
    return Rg, tg, R, t


@pytest.mark.parametrize("seed", [0, 1])
def test_global_rigid_motion_closed_form(tiny_problem, seed):
    P = tiny_problem
    Rg, tg, R, t = _global_rigid(P, seed)
    v = nr.warp(P, R, t)
    ref = P.base @ Rg.T + tg
    # the stored weights are FP32, so sum_s w_is = 1 only to within rounding
    wsum_err = np.abs(P.bind_w.sum(1) - 1.0).max()
    bound = 2.0 * (wsum_err + 1e-15) * np.linalg.norm(ref - P.base, axis=1).max() + 1e-14
    assert wsum_err < 1e-6
    assert np.abs(v - ref).max() <= bound
    assert np.abs(nr.arap_residuals(P, R, t)).max() < 1e-12


def test_arap_nonzero_for_relative_motion(tiny_problem):
    P = tiny_problem
    R, t = nr.identity_params(P.n)
    t = t.copy()
    t[3] += [0.01, 0.0, 0.0]
    r = nr.arap_residuals(P, R, t)
    touched = (P.edges[:, 0] == 3) | (P.edges[:, 1] == 3)
    assert np.allclose(np.linalg.norm(r[touched], axis=1),
                       np.sqrt(P.w_arap * P.edge_s[touched]) * 0.01)
    assert np.abs(r[~touched]).max() == 0.0


def test_bilinear_integer_and_affine():
    rng = np.random.default_rng(2)
    img = rng.normal(size=(9, 11))
    yy, xx = np.mgrid[:9, :11]
    u = xx.ravel().astype(float)
    v = yy.ravel().astype(float)
    assert np.array_equal(nr.bilinear(img, u, v), img.ravel())
    aff = 0.3 + 0.02 * xx - 0.05 * yy
    uq = rng.uniform(0, 10, 200)
    vq = rng.uniform(0, 8, 200)
    assert np.allclose(nr.bilinear(aff, uq, vq), 0.3 + 0.02 * uq - 0.05 * vq, atol=1e-14)
    gx, gy = nr.central_differences(aff)
    assert np.allclose(gx, 0.02) and np.allclose(gy, -0.05)
    # clamp to edge
    assert nr.bilinear(img, np.array([-3.0]), np.array([100.0]))[0] == img[8, 0]


def test_central_differences_definition():
    img = np.arange(20, dtype=float).reshape(4, 5) ** 2
    gx, gy = nr.central_differences(img)
    assert gx[1, 2] == (img[1, 3] - img[1, 1]) / 2
    assert gx[1, 0] == img[1, 1] - img[1, 0] and gx[1, 4] == img[1, 4] - img[1, 3]
    assert gy[2, 1] == (img[3, 1] - img[1, 1]) / 2 and gy[0, 1] == img[1, 1] - img[0, 1]
