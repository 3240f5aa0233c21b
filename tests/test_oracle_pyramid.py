"""Pins for the photometric pyramid of the oracle (oracle/pyramid.py and its
use in oracle.nonrigid / oracle.surface):

* the Gaussian taps: the size-to-width rule in closed form, unit sum,
  symmetry, the ratio of neighbouring taps;
* the blur against SciPy's Gaussian filter (clamp-to-edge mode, the same
  radius), and on constant and affine images, which a symmetric normalised
  kernel leaves unchanged away from the border;
* the box downsampling against a block-by-block loop on ragged sizes;
* the level coordinates: on an affine image every level, sampled at a
  full-resolution coordinate, returns the image's own value and gradient
  (a wrong centre offset or a missing 1/d fails this);
* the per-iteration level schedule;
* the Jacobian at every level against central finite differences on an
  affine image, and a planted mistake (the 1/d gradient scale dropped) that
  the same check catches;
* the finest level without blur reproduces the raw-image path exactly.
"""
import copy

import numpy as np
import pytest
from scipy import ndimage

from oracle import nonrigid as nr
from oracle import pyramid as pyr


def test_taps_closed_form():
    for k, sigma in ((15, 2.6), (9, 1.7), (3, 0.8), (5, 1.1)):
        w = pyr.gaussian_taps(k)
        r = (k - 1) // 2
        assert len(w) == k and np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
        assert np.array_equal(w, w[::-1])
        # neighbouring taps differ by exp(-(2i+1) / (2 sigma^2))
        i = np.arange(0, r)
        assert np.allclose(w[r + i + 1] / w[r + i], np.exp(-(2 * i + 1) / (2 * sigma ** 2)), rtol=1e-13)
    assert np.array_equal(pyr.gaussian_taps(1), [1.0])
    with pytest.raises(ValueError):
        pyr.gaussian_taps(4)


@pytest.mark.parametrize("k", [3, 9, 15])
def test_blur_matches_scipy(k):
    rng = np.random.default_rng(k)
    img = rng.uniform(size=(23, 37, 3))
    r = (k - 1) // 2
    sigma = 0.3 * (r - 1) + 0.8
    ref = ndimage.gaussian_filter1d(img, sigma, axis=1, mode="nearest", radius=r)
    ref = ndimage.gaussian_filter1d(ref, sigma, axis=0, mode="nearest", radius=r)
    assert np.abs(pyr.blur(img, k) - ref).max() <= 1e-14


def test_blur_constant_and_affine():
    H, W = 40, 52
    c = np.full((H, W, 3), 0.37)
    assert np.abs(pyr.blur(c, 15) - c).max() <= 1e-15
    yy, xx = np.mgrid[:H, :W].astype(np.float64)
    aff = np.stack([0.2 + 0.01 * xx - 0.003 * yy, 0.5 - 0.002 * xx + 0.004 * yy, 0.1 + 0.001 * xx], -1)
    b = pyr.blur(aff, 9)
    assert np.abs(b[4:-4, 4:-4] - aff[4:-4, 4:-4]).max() <= 1e-14
    # at the border the clamp bends it
    assert np.abs(b[0, 10] - aff[0, 10]).max() > 1e-4


@pytest.mark.parametrize("shape,d", [((17, 23), 4), ((16, 16), 4), ((9, 31), 2), ((1, 5), 4), ((6, 7), 1)])
def test_box_downsample(shape, d):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    img = rng.uniform(size=shape + (3,))
    out = pyr.box_downsample(img, d)
    assert out.shape == (-(-shape[0] // d), -(-shape[1] // d), 3)
    assert np.abs(out - pyr.box_downsample_brute(img, d)).max() <= 1e-15


def test_level_schedule():
    assert [pyr.level_of(g, 3) for g in range(5)] == [0, 1, 2, 2, 2]
    assert [pyr.level_of(g, 2) for g in range(3)] == [1, 2, 2]
    assert [pyr.level_of(g, 1) for g in range(2)] == [2, 2]
    assert pyr.level_of(0, 0) is None


def _affine_problem(P, ksize=(15, 9, 3)):
    Q = copy.copy(P)
    yy, xx = np.mgrid[:P.H, :P.W].astype(np.float64)
    Q.rgb = np.stack([0.5 + 0.004 * xx - 0.002 * yy, 0.3 - 0.003 * xx + 0.005 * yy,
                      0.4 + 0.001 * xx + 0.001 * yy], axis=-1)
    Q.dt = 2.0 + 0.05 * xx + 0.03 * yy
    Q._grad_rgb = None
    Q._grad_dt = None
    Q.pyr_ksize = ksize
    return Q


@pytest.mark.parametrize("j", [0, 1, 2])
def test_level_coordinates_on_affine_image(tiny_problem, j):
    Q = _affine_problem(tiny_problem)
    Q.level = j
    d = pyr.FACTORS[j]
    r = (Q.pyr_ksize[j] - 1) // 2
    m = d * (r + 2)          # far enough from the border for the clamp
    rng = np.random.default_rng(j)
    u = rng.uniform(m, Q.W - 1 - m, 200)
    w = rng.uniform(m, Q.H - 1 - m, 200)
    I, G = nr.photo_sample(Q, u, w, grad=True)
    a = np.array([0.5, 0.3, 0.4]) + np.outer(u, [0.004, -0.003, 0.001]) + np.outer(w, [-0.002, 0.005, 0.001])
    assert np.abs(I - a).max() <= 1e-13
    assert np.abs(G[:, :, 0] - [0.004, -0.003, 0.001]).max() <= 1e-13
    assert np.abs(G[:, :, 1] - [-0.002, 0.005, 0.001]).max() <= 1e-13
    Q.level = None
    assert np.abs(nr.photo_sample(Q, u, w) - a).max() <= 1e-13


def _fd_check(P, R, t, h=1e-6):
    """max |J - FD| / max |FD| over the photometric rows, decisions frozen."""
    vr = nr.vertex_residuals(P, R, t)
    on = vr["photo_on"]
    F, J = nr.linearise(P, R, t)
    n_p = 3 * int(on.sum())
    Jp = J.toarray()[:n_p]
    cols = []
    for c in range(6 * P.n):
        dp = np.zeros(6 * P.n)
        dp[c] = h
        Rp, tp = nr.apply_update(R, t, dp)
        Rm, tm = nr.apply_update(R, t, -dp)
        fp = nr.vertex_residuals(P, Rp, tp)
        fm = nr.vertex_residuals(P, Rm, tm)
        assert np.array_equal(fp["photo_on"], on) and np.array_equal(fm["photo_on"], on)
        cols.append((fp["photo"][on].ravel() - fm["photo"][on].ravel()) / (2 * h))
    Jfd = np.stack(cols, axis=1)
    return np.abs(Jp - Jfd).max() / np.abs(Jfd).max()


@pytest.mark.parametrize("j", [0, 1, 2])
def test_jacobian_fd_per_level(tiny_problem, j):
    # kernel size 1: the levels of an affine image are affine up to the border
    Q = _affine_problem(tiny_problem, ksize=(1, 1, 1))
    Q.level = j
    rng = np.random.default_rng(7 + j)
    R = nr.so3_exp(rng.normal(scale=0.03, size=(Q.n, 3)))
    t = rng.normal(scale=0.003, size=(Q.n, 3))
    assert _fd_check(Q, R, t) <= 1e-7


def test_planted_gradient_scale_fails(tiny_problem, monkeypatch):
    Q = _affine_problem(tiny_problem, ksize=(1, 1, 1))
    Q.level = 0
    rng = np.random.default_rng(9)
    R = nr.so3_exp(rng.normal(scale=0.03, size=(Q.n, 3)))
    t = rng.normal(scale=0.003, size=(Q.n, 3))
    orig = nr.photo_sample

    def no_scale(P, u, v, grad=False):
        out = orig(P, u, v, grad)
        if grad and P.level is not None:
            return out[0], out[1] * pyr.FACTORS[P.level]
        return out

    monkeypatch.setattr(nr, "photo_sample", no_scale)
    assert _fd_check(Q, R, t) > 1e-2


def test_raw_image_path_unchanged(tiny_scene, tiny_graph):
    """Without a pyramid the solve samples the raw image (level None)."""
    a = nr.solve_scene(tiny_scene, graph=tiny_graph, n_gn=2, n_pcg=3)
    assert a["problem"].level is None
    b = nr.solve_scene(tiny_scene, graph=tiny_graph, n_gn=2, n_pcg=3, pyr_levels=3)
    assert b["problem"].level == 2
    assert a["hist"][0]["energy"] != b["hist"][0]["energy"]


def test_finest_level_without_blur_is_the_raw_image(tiny_problem):
    """Factor 1 and one tap: level 2 is the frame itself, so sampling it
    reproduces the raw-image path exactly (values and gradients)."""
    Q = copy.copy(tiny_problem)
    Q.pyr_ksize = (15, 9, 1)
    rng = np.random.default_rng(3)
    u = rng.uniform(0, Q.W - 1, 300)
    w = rng.uniform(0, Q.H - 1, 300)
    Q.level = None
    I0, G0 = nr.photo_sample(Q, u, w, grad=True)
    Q.level = 2
    I2, G2 = nr.photo_sample(Q, u, w, grad=True)
    assert np.array_equal(I0, I2) and np.array_equal(G0, G2)
    assert np.array_equal(pyr.level_image(Q.rgb, 2, Q.pyr_ksize), Q.rgb)
