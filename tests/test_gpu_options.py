"""All options of the per-frame path together, end to end on the GPU against
the oracle: the distance transform computed on the device (frame uploaded
without one), the photometric pyramid (3 levels, one Gauss-Newton step per
level), the robust colour kernel sigma_c and the body-part mask, in the
paper's surface stage (3 GN x 4 PCG) on the body capture.

Bound: as each option's own end-to-end test, max(1e-4, 2 x the oracle's FP32
rounding band over 8 rounded runs) of the final energy and of every step's
energy, vertices within max(1e-4 x diagonal, 2 x band); the final pruning
and masking decisions may differ on at most max(2, 1%) vertices each, and
each such vertex moves the final energy by its own term (added to the bound).
"""
import copy

import numpy as np
import pytest

import synth
from gpu_helpers import report, surface_rounding_band
from oracle import dt as odt
from oracle import parts as oparts
from oracle import surface as osf

pytestmark = pytest.mark.gpu

FLAG_PRUNED, FLAG_MASKED = 16, 32


def _gap_sigma(d, quantile):
    v = np.sort(d[np.isfinite(d)])
    k = min(max(int(quantile * len(v)), 1), len(v) - 1)
    assert v[k] - v[k - 1] > 1e-6
    return float(np.float32(0.5 * (v[k - 1] + v[k])))


def test_surface_all_options_end_to_end():
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    body = synth.make_scene("body")
    scene = copy.copy(body)
    scene.dt = odt.distance_transform(body.mask)        # what the device computes
    sk = body.skeleton
    VS = np.asarray(body.meta["V_posed"], np.float32)
    V = VS.astype(np.float64)
    rng = np.random.default_rng(5)
    c = V.mean(0)
    V0 = (V + 0.004 * np.sin((V - c) @ rng.normal(size=(3, 3)) * 6.0)).astype(np.float32)
    vp = oparts.vertex_parts(sk["skin_idx"], sk["skin_w"], sk["bone_part"])
    cam = body.cam
    mask = oparts.part_mask(VS, body.F, cam.f, cam.cx, cam.cy, cam.W, cam.H, vp, 10, sk["torso_part"])
    # sigma_c between two colour distances of the first step (level 0)
    P0 = osf.problem_from_scene(scene, base32=VS)
    osf.frame_decisions(P0, V0)
    P0.pyr_levels, P0.level = 3, 0
    r0 = osf.residuals(P0, V0.astype(np.float64))
    d = np.linalg.norm(r0["photo"], axis=1) / np.sqrt(P0.w_photo)
    sigma = _gap_sigma(d[r0["photo_on"]], 0.9)

    ctx = Context(0)
    setup_scene(ctx, body)
    ctx.upload_frame(body.rgb, None, body.mask)          # the device distance transform
    dt_gpu, _ = ctx.read_frame()
    assert np.array_equal(dt_gpu, scene.dt)
    ctx.set_params(pyr_levels=3, sigma_c=sigma)
    ctx.set_body_parts(sk["bone_part"], sk["torso_part"], 10)
    ctx.set_rest_geometry(VS)
    ctx.set_surface(V0)
    stats = ctx.solve_surface()
    Vg, flags = ctx.read_surface(flags=True)
    kw = dict(base32=VS, V0=V0, sigma_c=sigma, pyr_levels=3, part_mask=mask, vpart=vp)
    ref, band_E, band_V = surface_rounding_band(scene, n_runs=8, **kw)
    P = ref["problem"]
    e_gpu, e_ref = stats["e_total"], ref["e1"]["total"]
    diag = np.linalg.norm(body.V.max(0) - body.V.min(0))
    dv = float(np.abs(Vg.astype(np.float64) - ref["V"]).max())
    e_hist = np.array(stats["e_gn"])
    e_hist_ref = np.array([h["energy"] for h in ref["hist"]])
    # final decisions of the two solves and the terms of the vertices they differ on
    rs = osf.residuals(P, ref["V"])
    masked = (flags & FLAG_MASKED) != 0
    pruned = (flags & FLAG_PRUNED) != 0
    flip_m = masked != (oparts.masked(P, ref["V"]) & P.inB)
    u = rs["u"]
    inimg = (u >= 0) & (u <= P.W - 1) & (rs["w"] >= 0) & (rs["w"] <= P.H - 1)
    flip_p = pruned != (P.vis & inimg & ~rs["photo_on"])
    Q = copy.copy(P)
    Q.part_mask = None
    Q.sigma_c = 0.0
    rq = osf.residuals(Q, ref["V"])
    e_flip = float((rq["sil"][flip_m] ** 2).sum() + (rq["photo"][flip_p] ** 2).sum())
    report("options_e2e_surface", e_gpu=e_gpu, e_ref=e_ref, rel=abs(e_gpu - e_ref) / e_ref,
           band_E_rel=band_E / e_ref, dv_over_diag=dv / diag, hist_rel=np.abs(e_hist - e_hist_ref).max() / e_hist_ref.max(),
           n_pruned=int(pruned.sum()), n_masked=int(masked.sum()), flips_p=int(flip_p.sum()),
           flips_m=int(flip_m.sum()), e_flip_rel=e_flip / e_ref, sigma=sigma)
    assert stats["pcg_iters"] == [h["pcg_iters"] for h in ref["hist"]]
    assert pruned.sum() > 0 and masked.sum() > 0
    assert flip_m.sum() <= max(2, P.inB.sum() // 100)
    assert flip_p.sum() <= max(2, P.vis.sum() // 100)
    assert abs(e_gpu - e_ref) <= max(1e-4 * e_ref, 2.0 * band_E) + e_flip
    assert np.abs(e_hist - e_hist_ref).max() <= max(1e-4 * e_hist_ref.max(), 2.0 * band_E) + e_flip
    assert dv <= max(1e-4 * diag, 2.0 * band_V)
    ctx.close()
