"""Pins for the body-part mask of the silhouette term (oracle/parts.py):

* vertex parts: the heaviest bone with the first of equal weights; on the
  synthetic body every vertex lands in the part of the capsule it belongs to;
* triangle labels: the majority rule on hand cases;
* the label image from a hand-made z-buffer;
* the dilation against a pixel-by-pixel brute force, against SciPy's exact
  distance transform for a single part, at the radius boundary, and the
  torso's precedence in a gap between two parts;
* the pixel lookup's FP32 rounding at half-pixel coordinates;
* the energy: the masked silhouette residuals are exactly the ones dropped.
"""
import copy

import numpy as np
import pytest
from scipy import ndimage

import synth
from oracle import nonrigid as nr
from oracle import parts as op

NONE = op.NONE


def test_vertex_parts_first_maximum():
    idx = np.array([[3, 1, 0, 0], [2, 4, 0, 0], [5, 5, 5, 5]])
    w = np.array([[0.5, 0.5, 0, 0], [0.2, 0.8, 0, 0], [0.25, 0.25, 0.25, 0.25]], np.float32)
    bone_part = np.array([9, 8, 7, 6, 5, 4])
    assert list(op.vertex_parts(idx, w, bone_part)) == [6, 5, 4]


def test_body_vertices_follow_their_capsule():
    s = synth.make_scene("body")
    sk = s.skeleton
    vp = op.vertex_parts(sk["skin_idx"], sk["skin_w"], sk["bone_part"])
    # capsules: torso, head, l upper arm, l forearm, r upper arm, r forearm,
    # l thigh, l shin, r thigh, r shin
    cap_part = np.array([0, 1, 2, 2, 3, 3, 4, 4, 5, 5])
    assert np.array_equal(vp, cap_part[sk["segment"]])


def test_triangle_labels():
    F = np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8], [9, 10, 11], [12, 13, 14]])
    vp = np.array([1, 1, 2, 4, 3, 3, 5, 6, 7, 2, 3, 2, 8, 8, 8], np.uint8)
    assert list(op.triangle_labels(F, vp)) == [1, 3, 5, 2, 8]


def test_label_image():
    F = np.array([[0, 1, 2], [2, 3, 4]])
    vp = np.array([1, 1, 2, 3, 3], np.uint8)
    z = np.full((2, 3), np.uint64(0xFFFFFFFFFFFFFFFF))
    z[0, 0] = (np.uint64(1234) << np.uint64(32)) | np.uint64(1)
    z[1, 2] = (np.uint64(77) << np.uint64(32)) | np.uint64(0)
    lab = op.label_image(z, F, vp)
    assert lab.tolist() == [[3, NONE, NONE], [NONE, NONE, 1]]


@pytest.mark.parametrize("seed,R,torso", [(0, 2, 0), (1, 3, -1), (2, 4, 1), (3, 0, 0), (4, 3, 2)])
def test_dilate_matches_brute_force(seed, R, torso):
    rng = np.random.default_rng(seed)
    raw = np.full((19, 23), NONE, np.uint8)
    pick = rng.uniform(size=raw.shape) < 0.04
    raw[pick] = rng.integers(0, 4, size=int(pick.sum()))
    assert np.array_equal(op.dilate(raw, R, torso), op.dilate_brute(raw, R, torso))


def test_dilate_single_part_is_the_distance_ball():
    yy, xx = np.mgrid[:64, :80]
    raw = np.full((64, 80), NONE, np.uint8)
    raw[((yy - 30) ** 2 + (xx - 33) ** 2 <= 81) | ((yy - 10) // 3 == (xx - 50) // 3)] = 2
    d = ndimage.distance_transform_edt(raw == NONE)
    out = op.dilate(raw, 10, 0)
    assert np.array_equal(out == 2, d <= 10.0)
    assert np.array_equal(out == NONE, d > 10.0)


def test_dilate_radius_boundary():
    raw = np.full((21, 21), NONE, np.uint8)
    raw[10, 10] = 4
    out = op.dilate(raw, 3, 0)
    assert out[10, 13] == 4 and out[12, 12] == 4       # d^2 = 9, 8
    assert out[13, 11] == NONE and out[10, 14] == NONE  # d^2 = 10, 16


def test_torso_precedence_in_a_gap():
    raw = np.full((20, 40), NONE, np.uint8)
    raw[:, :10] = 0            # torso
    raw[:, 16:] = 2            # an arm 6 px away
    out = op.dilate(raw, 10, 0)
    assert (out[:, 10:16] == 0).all()          # the gap closes with the torso label
    out2 = op.dilate(raw, 10, -1)              # without precedence: the nearer part
    assert (out2[:, 10:13] == 0).all() and (out2[:, 13:16] == 2).all()


def test_lookup_rounding():
    class _P:
        f, cx, cy = 1.0, 0.0, 0.0
        part_mask = np.array([[0, 1, 2, 3, 4, 5]], np.uint8)
        vpart = np.array([2, 2, 2, 2], np.uint8)
    X = np.array([2.5, np.nextafter(np.float32(2.5), np.float32(0)), 1.49, 5.0])
    V = np.stack([X, np.zeros(4), np.ones(4)], 1)
    m = op.masked(_P, V)
    # 2.5 -> pixel 3 (label 3: masked); just below 2.5 -> pixel 2 (own part)
    assert m.tolist() == [True, False, True, True]


def test_energy_drops_exactly_the_masked_rows(tiny_problem):
    P = tiny_problem
    rng = np.random.default_rng(5)
    R = nr.so3_exp(rng.normal(scale=0.03, size=(P.n, 3)))
    t = rng.normal(scale=0.003, size=(P.n, 3))
    vr0 = nr.vertex_residuals(P, R, t)
    Q = copy.copy(P)
    Q.part_mask = np.full((P.H, P.W), NONE, np.uint8)
    Q.part_mask[:, : P.W // 2] = 1          # left half belongs to another part
    Q.vpart = np.zeros(len(P.base), np.uint8)
    vr = nr.vertex_residuals(Q, R, t)
    m = op.masked(Q, vr0["v"])
    assert (m & vr0["sil_on"]).sum() > 0 and (~m & vr0["sil_on"]).sum() > 0
    assert np.array_equal(vr["sil_on"], vr0["sil_on"] & ~m)
    e0, e1 = nr.energy(P, R, t), nr.energy(Q, R, t)
    assert np.isclose(e0["sil"] - e1["sil"], float((vr0["sil"][m] ** 2).sum()), rtol=1e-12)
    assert e0["photo"] == e1["photo"] and e0["arap"] == e1["arap"]
