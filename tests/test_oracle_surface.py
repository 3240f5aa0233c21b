"""Pins for the oracle's per-vertex surface stage (oracle/surface.py).

* the one-ring against the Euler characteristic of closed capsules;
* the E_smooth / E_edge sums against a plain double loop over i and
  j in N_i on a tetrahedron, written from the energy's definition;
* invariances: E_smooth vanishes under a translation of V^S, E_edge under a
  rigid motion of the template, the temporal terms at a constant history;
* the assembled Jacobian against central finite differences of the residual
  vector on an affine image (bilinear sampling and central differences are
  exact there), every block separately, and a planted mistake failing it;
* with only the quadratic terms (smooth, velocity, acceleration) one
  Gauss-Newton step solved to convergence lands on the minimiser of the
  weighted graph Laplacian system built by scipy.sparse.csgraph;
* displacement warping: the blended rotation reduces to the bone's own for
  one bone, commutes with a global rotation, is the half-way rotation for
  two opposite bones, and a same-pose round trip returns the surface.
"""
import copy

import numpy as np
import pytest
from scipy.sparse import csgraph, coo_matrix, identity, kron
from scipy.sparse.linalg import spsolve

from oracle import nonrigid as nr
from oracle import surface as sf
from synth import capsule_mesh, make_scene


def _tet_problem(material=(1.0, 0.2, 0.5, 2.0)):
    V = np.array([[0.0, 0.0, 3.0], [0.1, 0.0, 3.0], [0.0, 0.1, 3.0], [0.0, 0.0, 3.1]])
    T = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]])
    img = np.zeros((8, 8, 3))
    P = sf.SurfaceProblem(base=V, tpl=V, albedo=np.zeros((4, 3)), material=np.array(material), tris=T,
                          f=10.0, cx=3.5, cy=3.5, W=8, H=8, rgb=img, dt=np.zeros((8, 8)),
                          mask=np.zeros((8, 8), bool), w_photo=0.0, w_sil=0.0, w_smooth=2.0, w_edge=3.0,
                          w_vel=0.5, w_acc=0.25)
    P.vis = np.zeros(4, bool)
    P.inB = np.zeros(4, bool)
    P.bsign = np.ones(4)
    return P


@pytest.mark.parametrize("rings,segments", [(4, 5), (10, 7), (40, 25)])
def test_one_ring_closed_capsule(rings, segments):
    V, F = capsule_mesh(0.3, 1.0, rings, segments)
    off, dst = sf.one_ring(len(V), F)
    src = sf.pair_sources(off)
    E2 = len(dst)
    assert E2 % 2 == 0
    assert len(V) - E2 // 2 + len(F) == 2                       # genus 0
    assert (src != dst).all()
    for i in range(len(V)):
        nb = dst[off[i]:off[i + 1]]
        assert (np.diff(nb) > 0).all()
        for j in nb:                                             # symmetric
            assert i in dst[off[j]:off[j + 1]]
    # closed manifold: a vertex has as many neighbours as incident triangles
    tri_count = np.bincount(np.asarray(F).ravel(), minlength=len(V))
    assert np.array_equal(np.diff(off), tri_count)


def test_regulariser_energies_by_double_loop():
    P = _tet_problem()
    rng = np.random.default_rng(0)
    V = P.base + rng.normal(scale=0.02, size=(4, 3))
    P.base = P.base + rng.normal(scale=0.01, size=(4, 3))      # V^S differs from the template
    P.__post_init__()
    P.vis = np.zeros(4, bool)
    P.inB = np.zeros(4, bool)
    P.bsign = np.ones(4)
    P.prev1 = P.base + 0.01
    P.prev2 = P.base - 0.02
    m = np.array([1.0, 0.2, 0.5, 2.0])
    nbrs = {0: [1, 2, 3], 1: [0, 2, 3], 2: [0, 1, 3], 3: [0, 1, 2]}
    es = ee = 0.0
    for i in range(4):
        for j in nbrs[i]:
            s = 0.5 * (m[i] + m[j])
            d = (V[i] - V[j]) - (P.base[i] - P.base[j])
            es += 2.0 * s / 3.0 * float(d @ d)
            ee += 3.0 * s / 3.0 * (np.linalg.norm(V[i] - V[j]) - np.linalg.norm(P.tpl[i] - P.tpl[j])) ** 2
    ev = 0.5 * sum(float((V[i] - P.prev1[i]) @ (V[i] - P.prev1[i])) for i in range(4))
    a = V - 2 * P.prev1 + P.prev2
    ea = 0.25 * float((a * a).sum())
    e = sf.energy(P, V)
    assert e["smooth"] == pytest.approx(es, rel=1e-13)
    assert e["edge"] == pytest.approx(ee, rel=1e-13)
    assert e["velocity"] == pytest.approx(ev, rel=1e-13)
    assert e["acceleration"] == pytest.approx(ea, rel=1e-13)
    # one previous frame only: V^{t-2} = V^{t-1}
    P.prev2 = None
    a1 = V - P.prev1
    assert sf.energy(P, V)["acceleration"] == pytest.approx(0.25 * float((a1 * a1).sum()), rel=1e-13)
    # no history: both temporal terms off
    P.prev1 = None
    e0 = sf.energy(P, V)
    assert e0["velocity"] == 0.0 and e0["acceleration"] == 0.0


def test_regulariser_invariances():
    scene = make_scene("tiny")
    P = sf.problem_from_scene(scene)
    P.vis = np.zeros(P.N, bool)
    P.inB = np.zeros(P.N, bool)
    P.bsign = np.ones(P.N)
    shift = np.array([0.03, -0.02, 0.05])
    assert sf.energy(P, P.base + shift)["smooth"] < 1e-24
    R = nr.so3_exp(np.array([[0.3, -0.2, 0.5]]))[0]
    Vr = P.tpl @ R.T + shift
    assert sf.energy(P, Vr)["edge"] < 1e-22
    assert sf.energy(P, Vr)["smooth"] > 1e-3                   # rotation is not free for E_smooth
    P.prev1 = P.prev2 = Vr
    e = sf.energy(P, Vr)
    assert e["velocity"] == 0.0 and e["acceleration"] == 0.0


def _affine(P):
    Q = copy.copy(P)
    yy, xx = np.mgrid[:P.H, :P.W].astype(np.float64)
    Q.rgb = np.stack([0.5 + 0.004 * xx - 0.002 * yy, 0.3 - 0.003 * xx + 0.005 * yy,
                      0.4 + 0.001 * xx + 0.001 * yy], axis=-1)
    Q.dt = 2.0 + 0.05 * xx + 0.03 * yy
    Q._grads = None
    return Q


def _stacked(P, V, on_p, on_s):
    r = sf.residuals(P, V)
    assert np.array_equal(r["photo_on"], on_p) and np.array_equal(r["sil_on"], on_s)
    out = [r["photo"][on_p].ravel(), r["sil"][on_s], r["smooth"].ravel(), r["edge"]]
    if P.prev1 is not None:
        out += [r["vel"].ravel(), r["acc"].ravel()]
    return np.concatenate(out)


def _fd_problem():
    scene = make_scene("tiny")
    P = sf.problem_from_scene(scene, prev1=scene.V + 0.004, prev2=scene.V - 0.003)
    rng = np.random.default_rng(3)
    V = P.base + rng.normal(scale=0.003, size=P.base.shape)
    sf.frame_decisions(P, V.astype(np.float32))
    assert P.vis.sum() > 100 and P.inB.sum() > 10 and (P.bsign < 0).sum() >= 0
    return _affine(P), V


def test_jacobian_matches_finite_differences():
    P, V = _fd_problem()
    F, J = sf.linearise(P, V, directions=False)
    r = sf.residuals(P, V)
    on_p, on_s = r["photo_on"], r["sil_on"]
    assert np.allclose(F, _stacked(P, V, on_p, on_s), rtol=0, atol=0)
    rng = np.random.default_rng(4)
    cols = rng.choice(3 * P.N, 60, replace=False)
    h = 1e-6
    Jd = J.tocsc()
    for c in cols:
        Vp, Vm = V.copy(), V.copy()
        Vp.flat[c] += h
        Vm.flat[c] -= h
        fd = (_stacked(P, Vp, on_p, on_s) - _stacked(P, Vm, on_p, on_s)) / (2 * h)
        col = Jd[:, c].toarray().ravel()
        assert np.abs(fd - col).max() <= 1e-6 * max(1.0, np.abs(col).max()), c


def test_planted_mistake_fails_the_fd_check(monkeypatch):
    """Drop the reverse-end block of E_edge: the FD check must see it."""
    P, V = _fd_problem()
    r = sf.residuals(P, V)
    on_p, on_s = r["photo_on"], r["sil_on"]
    F, J = sf.linearise(P, V, directions=False)
    # the edge rows of vertex 0's first pair, wrt the neighbour's columns
    j0 = int(P.dst[0])
    n_ph, n_si = 3 * on_p.sum(), on_s.sum()
    row = n_ph + n_si + 3 * len(P.src) + 0
    Jb = J.tolil()
    Jb[row, 3 * j0:3 * j0 + 3] = 0.0
    Jb = Jb.tocsc()
    c = 3 * j0
    h = 1e-6
    Vp, Vm = V.copy(), V.copy()
    Vp.flat[c] += h
    Vm.flat[c] -= h
    fd = (_stacked(P, Vp, on_p, on_s) - _stacked(P, Vm, on_p, on_s)) / (2 * h)
    assert np.abs(fd - Jb[:, c].toarray().ravel()).max() > 1e-3
    assert np.abs(fd - J.tocsc()[:, c].toarray().ravel()).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_quadratic_terms_reach_the_laplacian_minimiser():
    scene = make_scene("tiny")
    rng = np.random.default_rng(5)
    VS = scene.V.astype(np.float64) + rng.normal(scale=0.01, size=scene.V.shape)
    p1 = VS + rng.normal(scale=0.005, size=VS.shape)
    p2 = VS + rng.normal(scale=0.005, size=VS.shape)
    P = sf.problem_from_scene(scene, base32=VS.astype(np.float32),
                              weights=(0.0, 0.0, 1.0e3, 0.0, 25.0, 10.0), prev1=p1, prev2=p2)
    P.vis = np.zeros(P.N, bool)
    P.inB = np.zeros(P.N, bool)
    P.bsign = np.ones(P.N)
    V0 = P.base + rng.normal(scale=0.02, size=VS.shape)
    A, b, _, _ = sf.normal_equations(P, V0, directions=False)
    delta, info = nr.pcg(A, b, 3000)
    V1 = V0 + delta.reshape(-1, 3)
    # independent route: weighted Laplacian with c_ij = w_sm s_ij (1/|N_i| + 1/|N_j|)
    deg = np.diff(P.off).astype(np.float64)
    c = 1.0e3 * P.s * (1.0 / deg[P.src] + 1.0 / deg[P.dst])
    Wm = coo_matrix((c, (P.src, P.dst)), shape=(P.N, P.N)).tocsr()
    assert abs(Wm - Wm.T).max() < 1e-9
    L = csgraph.laplacian(Wm)
    M = kron(L, identity(3)) + (25.0 + 10.0) * identity(3 * P.N)
    rhs = kron(L, identity(3)) @ P.base.ravel() + 25.0 * p1.ravel() + 10.0 * (2 * p1 - p2).ravel()
    Vstar = spsolve(M.tocsc(), rhs).reshape(-1, 3)
    assert np.abs(V1 - Vstar).max() < 1e-8
    # the energy at the minimiser is below that of nearby points
    e_star = sf.energy(P, Vstar)["total"]
    for k in range(3):
        assert sf.energy(P, Vstar + rng.normal(scale=1e-4, size=Vstar.shape))["total"] > e_star


def _random_rotations(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return nr.so3_exp(rng.normal(scale=scale, size=(n, 3)))


def test_blend_rotations_special_cases():
    G = _random_rotations(6, 7)
    rng = np.random.default_rng(8)
    idx = rng.integers(0, 6, size=(50, 4))
    w = rng.uniform(0.0, 1.0, size=(50, 4))
    w /= w.sum(1, keepdims=True)
    # one bone with all the weight: that bone's rotation
    w1 = np.zeros((50, 4))
    w1[:, 0] = 1.0
    assert np.allclose(sf.blend_rotations(G, idx, w1), G[idx[:, 0]], atol=1e-12)
    # every slot on bones with the same rotation: that rotation
    Gs = np.tile(G[2], (6, 1, 1))
    assert np.allclose(sf.blend_rotations(Gs, idx, w), np.tile(G[2], (50, 1, 1)), atol=1e-12)
    # a rotation applied to every bone rotates the blend: blend(R G) = R blend(G)
    R = _random_rotations(1, 9)[0]
    Q = sf.blend_rotations(G, idx, w)
    assert np.allclose(sf.blend_rotations(R @ G, idx, w), R @ Q, atol=1e-12)
    # the result is a rotation; zero weights give the identity
    assert np.allclose(np.einsum("nji,njk->nik", Q, Q), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(Q), 1.0)
    assert np.allclose(sf.blend_rotations(G, idx, np.zeros((50, 4))), np.eye(3))
    # two bones at +-theta about one axis, equal weights: the identity
    # (the half-way rotation), and with weights (a, 1 - a) a rotation by
    # an angle strictly between the two
    axis = np.array([0.0, 0.0, 1.0])
    G2 = nr.so3_exp(np.stack([0.6 * axis, -0.6 * axis]))
    Qh = sf.blend_rotations(G2, np.array([[0, 1, 0, 0]]), np.array([[0.5, 0.5, 0.0, 0.0]]))
    assert np.allclose(Qh[0], np.eye(3), atol=1e-12)


def test_displacement_warping_round_trip():
    rng = np.random.default_rng(10)
    G = _random_rotations(5, 11)
    idx = rng.integers(0, 5, size=(40, 4))
    w = rng.uniform(size=(40, 4))
    w /= w.sum(1, keepdims=True)
    Q = sf.blend_rotations(G, idx, w)
    VS = rng.normal(size=(40, 3))
    V = VS + rng.normal(scale=0.01, size=(40, 3))
    dh = sf.record_displacement(V, VS, Q)
    # same pose: the surface comes back exactly
    assert np.allclose(sf.warped_start(VS, Q, dh), V, atol=1e-14)
    # lengths are preserved; a global extra rotation R rotates every displacement
    assert np.allclose(np.linalg.norm(dh, axis=1), np.linalg.norm(V - VS, axis=1))
    R = _random_rotations(1, 12)[0]
    Q2 = sf.blend_rotations(R @ G, idx, w)
    assert np.allclose(sf.warped_start(VS, Q2, dh) - VS, (V - VS) @ R.T, atol=1e-12)
