"""The silhouette distance transform computed on the device (lc_upload_frame
with dt = NULL) against the oracle (oracle/dt.py): bit-exact (integer
squared distances, one FP32 rounding of the square root), from capsule-sized
to 2048^2 frames, non-square frames, empty, full, single-pixel and noisy
silhouettes; and a solve on the device transform equals the solve on the
uploaded one bit for bit."""
import numpy as np
import pytest

import synth
from gpu_helpers import report
from oracle import dt as odt

pytestmark = pytest.mark.gpu


def _device_dt(mask, f=100.0):
    from paper_1810_02648_gb300 import Context
    H, W = mask.shape
    ctx = Context(0)
    ctx.set_camera(f, (W - 1) / 2.0, (H - 1) / 2.0, W, H)
    ctx.upload_frame(np.zeros((H, W, 3), np.float32), None, mask.astype(np.uint8))
    dt, m = ctx.read_frame()
    ctx.close()
    assert np.array_equal(m, mask.astype(np.uint8))
    return dt


def _blobs(H, W, seed, n=6):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[:H, :W]
    m = np.zeros((H, W), bool)
    for _ in range(n):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        a, b = rng.uniform(0.05, 0.3) * H, rng.uniform(0.05, 0.3) * W
        m |= ((yy - cy) / a) ** 2 + ((xx - cx) / b) ** 2 <= 1.0
    return m


@pytest.mark.parametrize("case", ["tiny", "body", "blobs_2048", "ragged", "noise", "empty", "full", "single"])
def test_device_distance_transform_bit_exact(case):
    if case in ("tiny", "body"):
        mask = synth.make_scene(case).mask
    elif case == "blobs_2048":
        mask = _blobs(2048, 2048, 1)
    elif case == "ragged":
        mask = _blobs(301, 517, 2)
    elif case == "noise":
        mask = np.random.default_rng(3).uniform(size=(97, 131)) < 0.55
    elif case == "empty":
        mask = np.zeros((64, 80), bool)
    elif case == "full":
        mask = np.ones((64, 80), bool)
    else:
        mask = np.zeros((50, 70), bool)
        mask[17, 41] = True
    got = _device_dt(mask)
    ref = odt.distance_transform(mask)
    report(f"dt_{case}", max_abs=float(np.abs(got - ref).max()), H=mask.shape[0], W=mask.shape[1])
    assert np.array_equal(got, ref)


def test_solve_on_device_transform_equals_uploaded():
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    scene = synth.make_scene("body")
    out = []
    for device_dt in (False, True):
        ctx = Context(0)
        setup_scene(ctx, scene, with_frame=False)
        ctx.upload_frame(scene.rgb, None if device_dt else scene.dt, scene.mask.astype(np.uint8),
                         scene.joints2d, scene.joints3d)
        st_p = ctx.solve_pose()
        st = ctx.solve_nonrigid()
        out.append((st_p["e_total"], st["e_total"], ctx.read_back()["V"]))
        ctx.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1] and np.array_equal(out[0][2], out[1][2])
