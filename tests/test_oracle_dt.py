"""Pins for the oracle's silhouette distance transform (oracle/dt.py):
SciPy's exact transform against brute force over every contour pixel on
random and structured small masks, the contour definition on hand-made
cases, and the empty / full / single-pixel special cases."""
import numpy as np
import pytest

from oracle import dt as odt


@pytest.mark.parametrize("seed,shape,p", [(0, (17, 23), 0.5), (1, (32, 32), 0.8), (2, (9, 40), 0.3),
                                          (3, (31, 1), 0.5), (4, (1, 29), 0.6)])
def test_scipy_matches_brute_force(seed, shape, p):
    rng = np.random.default_rng(seed)
    mask = rng.uniform(size=shape) < p
    assert np.array_equal(odt.squared_edt(mask), odt.squared_edt_brute(mask))


def test_disc_matches_brute_force_and_radius():
    yy, xx = np.mgrid[:64, :64]
    r2 = (yy - 31.3) ** 2 + (xx - 30.6) ** 2
    mask = r2 <= 20.0 ** 2
    d2 = odt.squared_edt(mask)
    assert np.array_equal(d2, odt.squared_edt_brute(mask))
    # far outside the disc the distance to the contour is |r - R| within a pixel
    far = r2 > 25.0 ** 2
    assert np.abs(np.sqrt(d2[far]) - (np.sqrt(r2[far]) - 20.0)).max() <= 1.0


def test_contour_definition():
    m = np.zeros((5, 6), bool)
    m[1:4, 1:5] = True
    c = odt.contour(m)
    expect = m.copy()
    expect[2, 2:4] = False          # the two pixels whose 4-neighbours are all foreground
    assert np.array_equal(c, expect)
    # foreground on the image border is contour
    full = np.ones((4, 5), bool)
    cf = odt.contour(full)
    assert cf[0].all() and cf[-1].all() and cf[:, 0].all() and cf[:, -1].all() and not cf[1:-1, 1:-1].any()


def test_special_cases():
    assert (odt.distance_transform(np.zeros((7, 9), bool)) == 0).all()
    full = np.ones((7, 9), bool)
    d2 = odt.squared_edt(full)
    yy, xx = np.mgrid[:7, :9]
    border = np.minimum(np.minimum(yy, 6 - yy), np.minimum(xx, 8 - xx))
    assert np.array_equal(d2, border ** 2)
    one = np.zeros((8, 8), bool)
    one[3, 5] = True
    y8, x8 = np.mgrid[:8, :8]
    assert np.array_equal(odt.squared_edt(one), (y8 - 3) ** 2 + (x8 - 5) ** 2)
    dtf = odt.distance_transform(one)
    assert dtf.dtype == np.float32 and dtf[3, 5] == 0.0 and dtf[0, 0] == np.float32(np.sqrt(np.float32(34.0)))
