"""Pins for the oracle's displacement warping of the graph stage
(oracle/surface.py ``graph_rest_params`` / ``graph_posed_params``): the
round trip through the rest pose, the identity when the pose does not
change, and rigid covariance: when every bone turns by the same rotation W
about the same point, the warped node parameters make the deformed surface
(warped by the oracle's own embedded-deformation warp) move rigidly with
the bones, v' = W v + c."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import nonrigid as onr
from oracle import surface as osf


def _rig(seed, N=60, J=5, n=12):
    rng = np.random.default_rng(seed)
    G = Rotation.from_rotvec(rng.normal(scale=0.6, size=(J, 3))).as_matrix()
    skin_idx = rng.integers(0, J, size=(N, 4))
    w = rng.uniform(0.1, 1.0, size=(N, 4))
    skin_w = w / w.sum(1, keepdims=True)
    node_vid = np.sort(rng.choice(N, size=n, replace=False))
    R = Rotation.from_rotvec(rng.normal(scale=0.2, size=(n, 3))).as_matrix()
    t = rng.normal(scale=0.05, size=(n, 3))
    return rng, G, skin_idx, skin_w, node_vid, R, t


def test_round_trip_and_identity():
    rng, G, si, sw, vid, R, t = _rig(1)
    Q = osf.blend_rotations(G, si, sw)
    Rr, tr = osf.graph_rest_params(R, t, vid, Q)
    R2, t2 = osf.graph_posed_params(Rr, tr, vid, Q)
    assert np.allclose(R2, R, atol=1e-13) and np.allclose(t2, t, atol=1e-14)
    # rest-pose parameters are rotations too
    assert np.allclose(np.einsum("nij,nkj->nik", Rr, Rr), np.eye(3), atol=1e-13)


def test_common_bone_rotation_moves_the_surface_rigidly():
    rng, G, si, sw, vid, R, t = _rig(2)
    N = len(si)
    W = Rotation.from_rotvec([0.3, -0.7, 0.4]).as_matrix()
    c = np.array([0.1, -0.2, 0.05])
    Q1 = osf.blend_rotations(G, si, sw)
    Q2 = osf.blend_rotations(np.einsum("ij,bjk->bik", W, G), si, sw)
    assert np.allclose(Q2, np.einsum("ij,njk->nik", W, Q1), atol=1e-12)
    Rr, tr = osf.graph_rest_params(R, t, vid, Q1)
    R2, t2 = osf.graph_posed_params(Rr, tr, vid, Q2)
    # the embedded graph on a base surface and on the same surface moved by (W, c)
    base = rng.normal(size=(N, 3))
    bind_idx = np.stack([rng.choice(len(vid), size=3, replace=False) for _ in range(N)])
    bw = rng.uniform(0.1, 1.0, size=(N, 3))
    bw /= bw.sum(1, keepdims=True)

    class P:
        pass
    p1, p2 = P(), P()
    for p, b in ((p1, base), (p2, base @ W.T + c)):
        p.base = b
        p.bind_idx = bind_idx
        p.bind_w = bw
        p.g = b[vid]
    v1 = onr.warp(p1, R, t)
    v2 = onr.warp(p2, R2, t2)
    assert np.allclose(v2, v1 @ W.T + c, atol=1e-12)
