"""Pins for the oracle's PCG and Gauss-Newton (CPU).

* Run to convergence, PCG equals a direct dense solve (numpy.linalg).
* After k iterations, CG's iterate minimises the A-norm error over the
  k-dimensional Krylov space of the preconditioned operator; that minimiser
  is computed independently by a projected direct solve.
* Gauss-Newton on a zero-residual problem converges quadratically.
"""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import nonrigid as nr


def _system(P, seed):
    rng = np.random.default_rng(seed)
    R = nr.so3_exp(rng.normal(scale=0.02, size=(P.n, 3)))
    t = rng.normal(scale=0.002, size=(P.n, 3))
    A, b, F, J = nr.normal_equations(P, R, t)
    A = (A + 1e-3 * sp.eye(A.shape[0])).tocsr()       # well-posed copy of J^T J
    return A, b


def test_pcg_converged_equals_direct_solve(tiny_problem):
    A, b = _system(tiny_problem, 0)
    x, info = nr.pcg(A, b, 4000)
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_pcg_krylov_optimality(tiny_problem, k):
    A, b = _system(tiny_problem, 1)
    Ad = A.toarray()
    d = np.diag(Ad)
    Minv = np.diag(1.0 / d)
    xs = np.linalg.solve(Ad, b)
    # Krylov basis of M^-1 A started from M^-1 b, orthonormalised
    vecs = [Minv @ b]
    for _ in range(k - 1):
        vecs.append(Minv @ (Ad @ vecs[-1]))
    Q, _ = np.linalg.qr(np.stack(vecs, 1))
    y = np.linalg.solve(Q.T @ Ad @ Q, Q.T @ b)
    x_ref = Q @ y
    x, info = nr.pcg(A, b, k)
    assert info["iters"] == k
    err_ref = np.sqrt((x_ref - xs) @ Ad @ (x_ref - xs))
    err = np.sqrt((x - xs) @ Ad @ (x - xs))
    assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    assert err <= err_ref * (1 + 1e-9)


def test_pcg_zero_rhs_and_breakdown():
    A = sp.csr_matrix(np.diag([1.0, 2.0, 3.0]))
    x, info = nr.pcg(A, np.zeros(3), 5)
    assert (x == 0).all() and info["iters"] == 0
    Aneg = sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]]))   # indefinite, positive diagonal
    x, info = nr.pcg(Aneg, np.array([1.0, -1.0]), 5)
    assert info["breakdown"] and info["iters"] == 0 and (x == 0).all()


def test_jacobi_zero_diagonal_rule():
    A = sp.csr_matrix(np.diag([2.0, 0.0, 4.0]))
    x, info = nr.pcg(A, np.array([2.0, 5.0, 4.0]), 3)
    assert np.allclose(x, [1.0, 0.0, 1.0])


def _zero_residual_problem(P):
    """Affine images, colours resampled at a rigidly moved surface, w_s = 0:
    the rigid motion is an exact zero of the energy."""
    Q = copy.copy(P)
    yy, xx = np.mgrid[:P.H, :P.W].astype(np.float64)
    Q.rgb = np.stack([0.5 + 0.004 * xx - 0.002 * yy, 0.3 - 0.003 * xx + 0.005 * yy,
                      0.4 + 0.001 * xx + 0.003 * yy], axis=-1)
    Q._grad_rgb = None
    Q._grad_dt = None
    Q.w_sil = 0.0
    Rg = nr.so3_exp(np.array([0.01, -0.02, 0.015]))[0]
    tg = np.array([0.003, -0.002, 0.001])
    R = np.tile(Rg, (P.n, 1, 1))
    t = P.g @ Rg.T + tg - P.g
    v = nr.warp(Q, R, t)
    u, w, valid, inimg = nr.project(Q, v)
    alb = Q.albedo.copy()
    alb[inimg] = nr.bilinear(Q.rgb, u[inimg], w[inimg])
    Q.albedo = alb
    return Q, R, t


def test_gauss_newton_quadratic_on_zero_residual(tiny_problem):
    Q, Rgt, tgt = _zero_residual_problem(tiny_problem)
    assert nr.energy(Q, Rgt, tgt)["total"] < 1e-24
    rng = np.random.default_rng(7)
    R = nr.so3_exp(rng.normal(scale=0.01, size=(Q.n, 3))) @ Rgt
    t = tgt + rng.normal(scale=0.001, size=(Q.n, 3))
    es = [nr.energy(Q, R, t)["total"]]
    for _ in range(4):
        R, t, _ = nr.gauss_newton(Q, R, t, 1, 3000)
        es.append(nr.energy(Q, R, t)["total"])
    assert es[-1] < 1e-16 * es[0]
    # quadratic: once small, each step roughly squares the relative energy
    assert es[2] / es[0] < (es[1] / es[0]) ** 1.5
