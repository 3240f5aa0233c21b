"""Finite-difference pins of the oracle's Jacobian and normal equations.

On images that are affine per channel, bilinear sampling is exact and central
differences equal the true gradient, so the assembled J must match a central
finite difference of the residual vector to FD accuracy.  A planted mistake
(the depth column of the projection derivative dropped) must fail the same
check.
"""
import copy

import numpy as np
import pytest

from oracle import nonrigid as nr


def _affine_problem(P):
    Q = copy.copy(P)
    H, W = P.H, P.W
    yy, xx = np.mgrid[:H, :W].astype(np.float64)
    Q.rgb = np.stack([0.5 + 0.004 * xx - 0.002 * yy, 0.3 - 0.003 * xx + 0.005 * yy,
                      0.4 + 0.001 * xx + 0.001 * yy], axis=-1)
    Q.dt = 2.0 + 0.05 * xx + 0.03 * yy
    Q._grad_rgb = None
    Q._grad_dt = None
    return Q


def _params(P, seed):
    rng = np.random.default_rng(seed)
    R = nr.so3_exp(rng.normal(scale=0.05, size=(P.n, 3)))
    t = rng.normal(scale=0.005, size=(P.n, 3))
    return R, t


def _stacked(P, R, t, on_p, on_s):
    vr = nr.vertex_residuals(P, R, t)
    assert np.array_equal(vr["photo_on"], on_p) and np.array_equal(vr["sil_on"], on_s)
    return np.concatenate([vr["photo"][on_p].ravel(), vr["sil"][on_s],
                           nr.arap_residuals(P, R, t).ravel()])


def _fd_jacobian(P, R, t, h=1e-6):
    vr = nr.vertex_residuals(P, R, t)
    on_p, on_s = vr["photo_on"], vr["sil_on"]
    cols = []
    for j in range(6 * P.n):
        d = np.zeros(6 * P.n)
        d[j] = h
        Rp, tp = nr.apply_update(R, t, d)
        Rm, tm = nr.apply_update(R, t, -d)
        cols.append((_stacked(P, Rp, tp, on_p, on_s) - _stacked(P, Rm, tm, on_p, on_s)) / (2 * h))
    Jfd = np.stack(cols, axis=1)
    # silhouette rows carry the direction sign b_i
    n_p = 3 * int(on_p.sum())
    n_s = int(on_s.sum())
    Jfd[n_p:n_p + n_s] *= P.bsign[on_s][:, None]
    return Jfd


def _check(P, R, t, rtol):
    F, J = nr.linearise(P, R, t)
    Jd = J.toarray()
    Jfd = _fd_jacobian(P, R, t)
    assert Jd.shape == Jfd.shape
    err = np.abs(Jd - Jfd)
    return err.max() <= rtol * np.abs(Jfd).max(), err.max() / np.abs(Jfd).max()


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobian_fd_affine_images(tiny_problem, seed):
    P = _affine_problem(tiny_problem)
    R, t = _params(P, seed)
    ok, rel = _check(P, R, t, 1e-7)
    assert ok, rel


def test_planted_mistake_fails_fd(tiny_problem, monkeypatch):
    P = _affine_problem(tiny_problem)
    R, t = _params(P, 0)
    real = nr.dproj

    def dropped_term(P_, v):
        D = real(P_, v)
        D[:, :, 2] = 0.0
        return D
    monkeypatch.setattr(nr, "dproj", dropped_term)
    ok, rel = _check(P, R, t, 1e-7)
    assert not ok and rel > 1e-3


def test_residual_vector_matches_energy(tiny_problem):
    P = tiny_problem
    R, t = _params(P, 3)
    F, _ = nr.linearise(P, R, t)
    e = nr.energy(P, R, t)
    assert np.isclose(F @ F, e["total"], rtol=1e-13)


def test_normal_equations_rhs_is_gradient(tiny_problem):
    """-J^T F is minus half the gradient of E on affine images (b_i = +1)."""
    P = _affine_problem(tiny_problem)
    P.bsign = np.ones_like(P.bsign)
    P.tris = None          # keep b_i = +1 (no direction update)
    R, t = _params(P, 4)
    A, b, F, J = nr.normal_equations(P, R, t)
    vr = nr.vertex_residuals(P, R, t)
    h = 1e-6
    rng = np.random.default_rng(5)
    for j in rng.choice(6 * P.n, 12, replace=False):
        d = np.zeros(6 * P.n)
        d[j] = h
        Ep = np.sum(_stacked(P, *nr.apply_update(R, t, d), vr["photo_on"], vr["sil_on"]) ** 2)
        Em = np.sum(_stacked(P, *nr.apply_update(R, t, -d), vr["photo_on"], vr["sil_on"]) ** 2)
        g = (Ep - Em) / (2 * h)
        # FD of a sum of squares loses ~1e-16 * E / h to cancellation
        assert np.isclose(-2.0 * b[j], g, rtol=1e-5, atol=1e-7 * max(1.0, Ep))
    # J^T J symmetric PSD
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T)
    assert np.linalg.eigvalsh(Ad).min() > -1e-9 * np.abs(Ad).max()
