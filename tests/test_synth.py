"""Pins for the seeded scene generator (CPU)."""
import numpy as np
import pytest

import synth
from synth import scenes


def _edges(F):
    a = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    return np.sort(a, axis=1)


def test_capsule_counts_closed_and_outward():
    V, F = synth.capsule_mesh(0.3, 1.0, 40, 25)
    assert V.shape == (1002, 3) and F.shape == (2000, 3)
    e, cnt = np.unique(_edges(F), axis=0, return_counts=True)
    assert (cnt == 2).all()                          # closed 2-manifold
    assert len(V) - len(e) + len(F) == 2             # sphere topology
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    exact = np.pi * 0.3 ** 2 * 0.4 + 4.0 / 3.0 * np.pi * 0.3 ** 3
    assert 0.95 * exact < vol < exact                # outward, inscribed polyhedron
    assert np.isclose(V[:, 1].max() - V[:, 1].min(), 1.0)


def test_body_counts():
    tpl = synth.body_template()
    assert tpl["V"].shape == (6020, 3) and tpl["F"].shape == (12000, 3)
    assert np.allclose(tpl["skin_w"].sum(1), 1.0)
    assert (tpl["skin_w"] >= 0).all()
    assert len(tpl["parents"]) == 23


def _brute_dt(mask):
    H, W = mask.shape
    m = mask.astype(bool)
    cont = []
    for y in range(H):
        for x in range(W):
            if not m[y, x]:
                continue
            border = x in (0, W - 1) or y in (0, H - 1)
            nb = [(y - 1, x), (y + 1, x), (y, x - 1), (y, x + 1)]
            if border or any(not m[j, i] for j, i in nb):
                cont.append((y, x))
    out = np.zeros((H, W))
    if not cont:
        return out
    c = np.array(cont, dtype=np.float64)
    for y in range(H):
        for x in range(W):
            out[y, x] = np.sqrt(((c - [y, x]) ** 2).sum(1)).min()
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_edt_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    m = np.zeros((24, 20), dtype=bool)
    for _ in range(3):
        y0, x0 = rng.integers(0, 18), rng.integers(0, 14)
        m[y0:y0 + rng.integers(3, 8), x0:x0 + rng.integers(3, 8)] = True
    assert np.array_equal(synth.contour_distance_transform(m), _brute_dt(m))


def test_edt_disc_and_empty():
    H = W = 64
    yy, xx = np.mgrid[:H, :W]
    r = np.hypot(xx - 31.5, yy - 31.5)
    m = r <= 20.0
    dt = synth.contour_distance_transform(m)
    assert np.abs(dt - np.abs(r - 20.0)).max() <= 1.5
    assert (synth.contour_distance_transform(np.zeros((8, 8), bool)) == 0).all()


def test_render_single_triangle():
    cam = synth.Camera(f=100.0, W=64, H=64)
    Z = 2.0
    # a screen-space triangle with vertices at known pixel positions
    px = np.array([[10.0, 10.0], [50.0, 12.0], [20.0, 50.0]])
    V = np.column_stack([(px[:, 0] - cam.cx) * Z / cam.f, (px[:, 1] - cam.cy) * Z / cam.f,
                         np.full(3, Z)])
    col = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    rgb, mask = synth.render(V, np.array([[0, 1, 2]]), col, cam)
    area = 0.5 * abs((50 - 10) * (50 - 10) - (12 - 10) * (20 - 10))
    assert abs(mask.sum() - area) < 0.6 * 130       # within a perimeter band
    assert np.allclose(rgb[10, 10], col[0]) and np.allclose(rgb[12, 50], col[1])
    assert np.allclose(rgb[mask].sum(1), 1.0)       # barycentric partition of unity


def test_albedo_range_and_determinism():
    V, _ = synth.capsule_mesh(0.3, 1.0, 10, 12)
    a = synth.value_noise_albedo(V, 3)
    assert a.min() >= 0.1 - 1e-12 and a.max() <= 0.9 + 1e-12
    assert np.array_equal(a, synth.value_noise_albedo(V, 3))
    assert not np.array_equal(a, synth.value_noise_albedo(V, 4))


def test_splitmix64_reference_values():
    # first outputs of splitmix64 seeded with 0 (Vigna's reference generator)
    st = np.uint64(0)
    got = []
    with np.errstate(over="ignore"):
        for i in range(3):
            got.append(int(scenes.splitmix64(np.array([st + np.uint64(0x9E3779B97F4A7C15) * np.uint64(i)],
                                                      dtype=np.uint64))[0]))
    assert got[0] == 0xE220A8397B1DCDAF
    assert got[1] == 0x6E789E6AA1B965F4
    assert got[2] == 0x06C45D188009454F


def test_ar1_frame_matches_the_sequence():
    """A frame generated on its own (blended-matrix field) equals the same
    frame of the serial sequence (per-control blend) up to rounding, and the
    AR(1) draws keep their stationary scale."""
    V, _ = synth.capsule_mesh(0.3, 1.0, 12, 10)
    seq = synth.ar1_sequence(V, 6, 20, 0.05, 0.01, seed=4)
    for i in (0, 3, 5):
        one = synth.ar1_frame(V, 20, 0.05, 0.01, seed=4, i=i)
        assert np.abs(one - seq[i]).max() <= 1e-12
    _, _, draws = synth.ar1_draws(V, 400, 50, 0.05, 0.01, seed=5)
    aa = np.stack([d[0] for d in draws])
    assert 0.045 < aa.std() < 0.055
    # lag-one correlation of the rotations: rho = 0.9
    r = (aa[1:] * aa[:-1]).mean() / (aa * aa).mean()
    assert 0.85 < r < 0.95
