"""GPU parity of the photometric pyramid (Sec. 3.4: a 3-level pyramid of the
input image, Gaussian blurred with kernel sizes 15, 9 and 3, one
Gauss-Newton iteration per level) against the FP64 oracle.

Tolerances:

* level images: FP32 box means of <= 16 pixels and <= 31 FP32 taps (each
  rounded once from FP64) against FP64: |gpu - ref| <= 4e-6 of the image's
  largest value;
* linearisation at each level, at identical FP32 inputs of the residual
  kernel (positions, projections and the level image the kernel samples):
  as without the pyramid (1e-5 per residual and per-vertex block, 1e-4 per
  node vector); the level coordinate (u - (d-1)/2) / d costs one FP32
  rounding of u;
* end to end (graph stage, 3 PCG iterations; surface stage, the paper's
  3 x 4): final and per-iteration energies and positions as strict as the
  raw-image end-to-end tests (1e-4, or twice the oracle's FP32 rounding
  band where that is larger).
"""
import numpy as np
import pytest

import synth
from gpu_helpers import (graph_from_gpu, oracle_problem, oracle_vertex_blocks, ragged_scene, random_params,
                         report, vec6)
from oracle import nonrigid as onr
from oracle import pyramid as opyr

pytestmark = pytest.mark.gpu


def _ctx(scene, **params):
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    ctx = Context(0)
    setup_scene(ctx, scene)
    if params:
        ctx.set_params(**params)
    return ctx


@pytest.fixture(scope="module")
def tiny():
    return synth.make_scene("tiny")


@pytest.fixture(scope="module")
def body():
    return synth.make_scene("body")


def _scenes(tiny, body):
    return {"tiny": tiny, "body": body, "ragged": ragged_scene(13, 11, 37, 3, side=70, shift=0.3)}


@pytest.mark.parametrize("case", ["tiny", "body", "ragged"])
@pytest.mark.parametrize("ksize", [(15, 9, 3), (5, 1, 7)])
def test_level_images(case, ksize, tiny, body):
    scene = _scenes(tiny, body)[case]
    # the pyramid is built when the parameters change after the frame ...
    ctx = _ctx(scene, pyr_levels=3, pyr_ksize=ksize)
    rgb = np.asarray(scene.rgb, dtype=np.float64)
    worst = 0.0
    for j in range(3):
        lvl = ctx.read_pyramid_level(j)
        ref = opyr.level_image(rgb, j, ksize)
        assert lvl.shape == ref.shape
        err = np.abs(lvl - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
    report(f"pyramid_levels_{case}_{'_'.join(map(str, ksize))}", rel=worst)
    assert worst <= 4e-6
    # ... and when a frame arrives with the pyramid on (bit-identical rebuild)
    before = [ctx.read_pyramid_level(j) for j in range(3)]
    ctx.upload_frame(scene.rgb, scene.dt, scene.mask)
    for j in range(3):
        assert np.array_equal(ctx.read_pyramid_level(j), before[j])
    ctx.close()


def test_level_availability(tiny):
    from paper_1810_02648_gb300 import LivecapError
    ctx = _ctx(tiny)
    with pytest.raises(LivecapError):
        ctx.read_pyramid_level(2)            # pyramid off
    ctx.set_params(pyr_levels=1)
    assert ctx.read_pyramid_level(2).shape == (tiny.cam.H, tiny.cam.W, 3)
    with pytest.raises(LivecapError):
        ctx.read_pyramid_level(1)            # only the finest level is built
    ctx.set_params(pyr_levels=2)
    assert ctx.read_pyramid_level(1).shape == ((tiny.cam.H + 1) // 2, (tiny.cam.W + 1) // 2, 3)
    with pytest.raises(LivecapError):
        ctx.set_params(pyr_ksize=(15, 8, 3))  # even size
    with pytest.raises(LivecapError):
        ctx.set_params(pyr_levels=4)
    ctx.close()


def _lin_level(scene, L, seed, tag):
    """Linearisation at Gauss-Newton step 0 with L levels: level j = 3 - L."""
    j = 3 - L
    ctx = _ctx(scene, pyr_levels=L)
    n = scene.n_nodes
    R, t = random_params(n, seed)
    ctx.set_node_params(R.reshape(n, 9), t)
    ctx.compute_visibility()
    lin = ctx.eval_linearization()
    g = ctx.read_graph()
    flags = ctx.read_visibility()["flags"]
    P = oracle_problem(scene, g, flags)
    P.tris = None
    P.pyr_levels, P.level = L, j
    # identical inputs: the residual kernel's level image is the GPU's FP32
    # one (checked against the FP64 level in test_level_images); differencing
    # a blurred FP32 image would otherwise magnify its rounding in the
    # gradients
    lvl = ctx.read_pyramid_level(j).astype(np.float64)
    P._pyr_cache = (P.rgb, {(tuple(int(k) for k in P.pyr_ksize), j): (lvl, onr.central_differences(lvl))})
    ref = oracle_vertex_blocks(P, lin["v"], lin["uv"])
    sp, ss = np.sqrt(P.w_photo), np.sqrt(P.w_sil)
    d_ph = np.abs(lin["r_photo"] - ref["r_photo"]) / np.maximum(np.abs(ref["r_photo"]), sp)
    d_si = np.abs(lin["r_sil"] - ref["r_sil"]) / np.maximum(np.abs(ref["r_sil"]), ss)
    scale = np.maximum(np.abs(ref["H"]).max(1), 1e-30)
    d_H = np.abs(lin["H"] - ref["H"]).max(1) / scale
    escale = np.maximum(np.abs(ref["e"]).max(1), np.sqrt(scale) * sp)
    d_e = np.abs(lin["e"] - ref["e"]).max(1) / escale
    e_ref = np.array([(ref["r_photo"] ** 2).sum(), (ref["r_sil"] ** 2).sum(),
                      (onr.arap_residuals(P, R.astype(np.float64), t.astype(np.float64)) ** 2).sum()])
    d_en = np.abs(lin["energy"] - e_ref) / np.maximum(e_ref, 1e-12)
    rhs, diag = ctx.eval_gradient()
    F, J = onr.linearise(P, R.astype(np.float64), t.astype(np.float64))
    JT = J.T.tocsr()
    rhs_ref = -(JT @ F)
    diag_ref = np.asarray((JT.multiply(JT)).sum(1)).ravel()
    p = np.random.default_rng(seed + 100).normal(size=6 * n).astype(np.float32)
    Ap = ctx.apply_jtj(p)
    Ap_ref = JT @ (J @ p.astype(np.float64))
    d_rhs = np.abs(vec6(rhs) - rhs_ref).max() / np.abs(rhs_ref).max()
    d_diag = np.abs(vec6(diag) - diag_ref).max() / np.abs(diag_ref).max()
    d_Ap = np.abs(vec6(Ap) - Ap_ref).max() / np.abs(Ap_ref).max()
    report(f"pyramid_lin_{tag}_L{L}", r_photo=d_ph.max(), r_sil=d_si.max(), H=d_H.max(), e=d_e.max(),
           energy=d_en.max(), rhs=d_rhs, diag=d_diag, jtjp=d_Ap, e_photo=float(lin["energy"][0]))
    assert d_ph.max() <= 1e-5 and d_si.max() <= 1e-5
    assert d_H.max() <= 1e-5 and d_e.max() <= 1e-5
    assert d_en.max() <= 1e-5
    assert d_rhs <= 1e-4 and d_diag <= 1e-4 and d_Ap <= 1e-4
    ctx.close()
    return lin


@pytest.mark.parametrize("L", [1, 2, 3])
def test_linearization_per_level_tiny(tiny, L):
    _lin_level(tiny, L, 31, "tiny")


@pytest.mark.parametrize("L", [1, 3])
def test_linearization_per_level_body(body, L):
    _lin_level(body, L, 32, "body")


def test_linearization_per_level_ragged():
    _lin_level(ragged_scene(13, 11, 37, 3, side=70, shift=0.3), 3, 33, "ragged")


def test_graph_end_to_end_tiny(tiny):
    from gpu_helpers import fp32_rounding_band
    ctx = _ctx(tiny, n_pcg=3, pyr_levels=3)
    stats = ctx.solve_nonrigid()
    out = ctx.read_back()
    graph = graph_from_gpu(ctx.read_graph())
    ref, band_E, band_V = fp32_rounding_band(tiny, graph, n_pcg=3, pyr_levels=3)
    e_gpu, e_ref = stats["e_total"], ref["e1"]["total"]
    diag = np.linalg.norm(tiny.V.max(0) - tiny.V.min(0))
    dv = float(np.abs(out["V"].astype(np.float64) - ref["v"]).max())
    e_hist = np.array(stats["e_gn"])
    e_hist_ref = np.array([h["energy"] for h in ref["hist"]])
    report("pyramid_e2e_graph_tiny", e_gpu=e_gpu, e_ref=e_ref, rel=abs(e_gpu - e_ref) / e_ref,
           band_E_rel=band_E / e_ref, dv_over_diag=dv / diag, band_V=band_V,
           hist_rel=np.abs(e_hist - e_hist_ref).max() / e_hist_ref.max())
    assert stats["pcg_iters"] == [h["pcg_iters"] for h in ref["hist"]]
    assert abs(e_gpu - e_ref) <= max(1e-4 * e_ref, 2.0 * band_E)
    assert np.abs(e_hist - e_hist_ref).max() <= max(1e-4 * e_hist_ref.max(), 2.0 * band_E)
    assert dv <= max(1e-4 * diag, 2.0 * band_V)
    ctx.close()


def test_surface_end_to_end_body(body):
    """The paper's schedule: 3 Gauss-Newton steps x 4 PCG, one per level."""
    from gpu_helpers import surface_rounding_band
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    VS = np.asarray(body.meta["V_posed"], dtype=np.float32)
    V = VS.astype(np.float64)
    rng = np.random.default_rng(3)
    c = V.mean(0)
    V0 = (V + 0.004 * np.sin((V - c) @ rng.normal(size=(3, 3)) * 6.0)).astype(np.float32)
    ctx = Context(0)
    setup_scene(ctx, body)
    ctx.set_params(pyr_levels=3)
    ctx.set_rest_geometry(VS)
    ctx.set_surface(V0)
    stats = ctx.solve_surface()
    Vg = ctx.read_surface()
    ref, band_E, band_V = surface_rounding_band(body, base32=VS, V0=V0, pyr_levels=3)
    e_gpu, e_ref = stats["e_total"], ref["e1"]["total"]
    diag = np.linalg.norm(body.V.max(0) - body.V.min(0))
    dv = float(np.abs(Vg.astype(np.float64) - ref["V"]).max())
    e_hist = np.array(stats["e_gn"])
    e_hist_ref = np.array([h["energy"] for h in ref["hist"]])
    report("pyramid_e2e_surface_body", e_gpu=e_gpu, e_ref=e_ref, rel=abs(e_gpu - e_ref) / e_ref,
           band_E_rel=band_E / e_ref, dv_over_diag=dv / diag, band_V=band_V,
           hist_rel=np.abs(e_hist - e_hist_ref).max() / e_hist_ref.max(), e0=ref["e0"]["total"])
    assert len(e_hist) == 3
    assert stats["pcg_iters"] == [h["pcg_iters"] for h in ref["hist"]]
    assert abs(e_gpu - e_ref) <= max(1e-4 * e_ref, 2.0 * band_E)
    assert np.abs(e_hist - e_hist_ref).max() <= max(1e-4 * e_hist_ref.max(), 2.0 * band_E)
    assert dv <= max(1e-4 * diag, 2.0 * band_V)
    ctx.close()
