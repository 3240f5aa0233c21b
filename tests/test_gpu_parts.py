"""GPU parity of the body-part mask of the silhouette term (Sec. 3.4) against
the oracle.

Integer work is bit-exact: the vertex parts, the label image of the rest
geometry V^S (the exact rasteriser), the dilated mask, and the MASKED
decisions of each linearisation at identical FP32 positions (the pixel is
decided from the FP32 projection, which both sides compute with the same
once-rounded operations).  With the mask on, the linearisation and the
end-to-end surface solve meet the tolerances of the unmasked tests.
"""
import copy

import numpy as np
import pytest

import synth
from gpu_helpers import (oracle_problem, oracle_vertex_blocks, random_params, report, surface_rounding_band,
                         vec6)
from oracle import nonrigid as onr
from oracle import parts as oparts
from oracle import surface as osf

pytestmark = pytest.mark.gpu

FLAG_MASKED = 32


@pytest.fixture(scope="module")
def body():
    return synth.make_scene("body")


@pytest.fixture(scope="module")
def body_parts(body):
    sk = body.skeleton
    vp = oparts.vertex_parts(sk["skin_idx"], sk["skin_w"], sk["bone_part"])
    VS = np.asarray(body.meta["V_posed"], np.float32)
    cam = body.cam
    mask_posed = oparts.part_mask(VS, body.F, cam.f, cam.cx, cam.cy, cam.W, cam.H, vp, 10, sk["torso_part"])
    mask_tpl = oparts.part_mask(body.V, body.F, cam.f, cam.cx, cam.cy, cam.W, cam.H, vp, 10, sk["torso_part"])
    return vp, VS, mask_posed, mask_tpl


def _ctx(scene):
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    ctx = Context(0)
    setup_scene(ctx, scene)
    sk = scene.skeleton
    ctx.set_body_parts(sk["bone_part"], sk["torso_part"], 10)
    return ctx


def _start(VS, seed=3):
    V = VS.astype(np.float64)
    rng = np.random.default_rng(seed)
    c = V.mean(0)
    return (V + 0.004 * np.sin((V - c) @ rng.normal(size=(3, 3)) * 6.0)).astype(np.float32)


def test_part_mask_bit_exact(body, body_parts):
    vp, VS, mask_posed, mask_tpl = body_parts
    ctx = _ctx(body)
    # graph stage: the rest geometry is the template
    ctx.compute_visibility()
    m, v = ctx.read_part_mask()
    assert np.array_equal(v, vp)
    assert np.array_equal(m, mask_tpl)
    # surface stage with the posed rest geometry V^S
    ctx.set_rest_geometry(VS)
    ctx.set_surface(_start(VS))
    ctx.surface_visibility()
    m2, _ = ctx.read_part_mask()
    assert np.array_equal(m2, mask_posed)
    report("parts_mask", labelled=int((m2 != 255).sum()), torso=int((m2 == 0).sum()))
    ctx.close()


def test_surface_linearization_masked(body, body_parts):
    vp, VS, mask_posed, _ = body_parts
    V0 = _start(VS)
    ctx = _ctx(body)
    ctx.set_rest_geometry(VS)
    ctx.set_surface(V0)
    ctx.surface_visibility()
    flags0 = ctx.read_visibility()["flags"]
    lin = ctx.surface_linearize()
    flags = ctx.read_visibility()["flags"]
    P = osf.problem_from_scene(body, base32=VS)
    P.vis = (flags0 & 1) != 0
    P.inB = (flags0 & 4) != 0
    P.bsign = np.where((flags & 8) != 0, -1.0, 1.0)
    P.part_mask, P.vpart = mask_posed, vp
    V = V0.astype(np.float64)
    rs = osf.residuals(P, V)
    masked = (flags & FLAG_MASKED) != 0
    ref_masked = oparts.masked(P, V0) & P.inB
    assert np.array_equal(masked, ref_masked)
    assert masked.sum() > 0
    assert not (rs["sil_on"] & masked).any()
    e_ref = osf.energy(P, V)
    e_vec = np.array([e_ref[k] for k in ("photo", "sil", "smooth", "edge", "velocity", "acceleration")])
    d_en = np.abs(lin["energy"] - e_vec) / np.maximum(np.abs(e_vec), 1e-12)
    A, b, F, J = osf.normal_equations(P, V, directions=False)
    JT = J.T.tocsr()
    diag_ref = np.asarray(JT.multiply(JT).sum(1)).ravel()
    d_rhs = np.abs(lin["rhs"].ravel() - b).max() / np.abs(b).max()
    d_diag = np.abs(lin["diag"].ravel() - diag_ref).max() / np.abs(diag_ref).max()
    p = np.random.default_rng(8).normal(size=V.shape).astype(np.float32)
    Ap = ctx.surface_apply_jtj(p)
    Ap_ref = A @ p.astype(np.float64).ravel()
    d_Ap = np.abs(Ap.ravel() - Ap_ref).max() / np.abs(Ap_ref).max()
    report("parts_surface_lin", masked=int(masked.sum()), n_B=int(P.inB.sum()), energy=d_en.max(), rhs=d_rhs,
           diag=d_diag, jtjp=d_Ap)
    assert d_en.max() <= 1e-5
    assert d_rhs <= 1e-4 and d_diag <= 1e-4 and d_Ap <= 1e-4
    # switching the mask off clears the flag at the next linearisation
    ctx.set_body_parts(None)
    ctx.surface_linearize()
    assert not (ctx.read_visibility()["flags"] & FLAG_MASKED).any()
    ctx.close()


def test_graph_linearization_masked(body, body_parts):
    vp, _, _, mask_tpl = body_parts
    ctx = _ctx(body)
    n = body.n_nodes
    R, t = random_params(n, 41, rot=0.08, trans=0.01)
    ctx.set_node_params(R.reshape(n, 9), t)
    ctx.compute_visibility()
    lin = ctx.eval_linearization()
    flags = ctx.read_visibility()["flags"]
    P = oracle_problem(body, ctx.read_graph(), flags)
    P.tris = None
    P.part_mask, P.vpart = mask_tpl, vp
    masked = (flags & FLAG_MASKED) != 0
    assert np.array_equal(masked, oparts.masked(P, lin["v"]) & P.inB)
    ref = oracle_vertex_blocks(P, lin["v"], lin["uv"])
    assert not (ref["sil_on"] & masked).any()
    ss = np.sqrt(P.w_sil)
    d_si = np.abs(lin["r_sil"] - ref["r_sil"]) / np.maximum(np.abs(ref["r_sil"]), ss)
    scale = np.maximum(np.abs(ref["H"]).max(1), 1e-30)
    d_H = np.abs(lin["H"] - ref["H"]).max(1) / scale
    rhs, diag = ctx.eval_gradient()
    F, J = onr.linearise(P, R.astype(np.float64), t.astype(np.float64))
    JT = J.T.tocsr()
    rhs_ref = -(JT @ F)
    d_rhs = np.abs(vec6(rhs) - rhs_ref).max() / np.abs(rhs_ref).max()
    report("parts_graph_lin", masked=int(masked.sum()), r_sil=d_si.max(), H=d_H.max(), rhs=d_rhs)
    assert d_si.max() <= 1e-5 and d_H.max() <= 1e-5 and d_rhs <= 1e-4
    ctx.close()


def test_surface_end_to_end_masked(body, body_parts):
    vp, VS, mask_posed, _ = body_parts
    V0 = _start(VS)
    ctx = _ctx(body)
    ctx.set_rest_geometry(VS)
    ctx.set_surface(V0)
    stats = ctx.solve_surface()
    Vg, flags = ctx.read_surface(flags=True)
    # the body's surface solve spreads by ~1e-4 of its energy under FP32
    # rounding; 8 rounded runs estimate that band
    ref, band_E, band_V = surface_rounding_band(body, base32=VS, V0=V0, part_mask=mask_posed, vpart=vp, n_runs=8)
    e_gpu, e_ref = stats["e_total"], ref["e1"]["total"]
    diag = np.linalg.norm(body.V.max(0) - body.V.min(0))
    dv = float(np.abs(Vg.astype(np.float64) - ref["V"]).max())
    e_hist = np.array(stats["e_gn"])
    e_hist_ref = np.array([h["energy"] for h in ref["hist"]])
    # the final decisions: a contour vertex within the two solves' distance of
    # a pixel boundary between two labels may be decided either way; each such
    # vertex moves the final energy by its silhouette term (evaluated with the
    # mask ignored, i.e. as the side that keeps it sees it)
    P = ref["problem"]
    masked = (flags & FLAG_MASKED) != 0
    flip = masked != (oparts.masked(P, ref["V"]) & P.inB)
    Q = copy.copy(P)
    Q.part_mask = None
    e_flip = float((osf.residuals(Q, ref["V"])["sil"][flip] ** 2).sum())
    report("parts_e2e_surface", e_gpu=e_gpu, e_ref=e_ref, rel=abs(e_gpu - e_ref) / e_ref,
           band_E_rel=band_E / e_ref, dv_over_diag=dv / diag, masked=int(masked.sum()), flips=int(flip.sum()),
           e_flip_rel=e_flip / e_ref)
    assert stats["pcg_iters"] == [h["pcg_iters"] for h in ref["hist"]]
    assert flip.sum() <= max(2, P.inB.sum() // 100)
    assert abs(e_gpu - e_ref) <= max(1e-4 * e_ref, 2.0 * band_E) + e_flip
    assert np.abs(e_hist - e_hist_ref).max() <= max(1e-4 * e_hist_ref.max(), 2.0 * band_E)
    assert dv <= max(1e-4 * diag, 2.0 * band_V)
    ctx.close()


def test_body_parts_arguments(body):
    from paper_1810_02648_gb300 import Context, LivecapError
    from synth import setup_scene
    tiny = synth.make_scene("tiny")
    ctx = Context(0)
    setup_scene(ctx, tiny)
    with pytest.raises(LivecapError):
        ctx.set_body_parts(np.zeros(23, np.int32), 0, 10)       # no skeleton
    ctx.close()
    ctx = _ctx(body)
    bp = body.skeleton["bone_part"]
    with pytest.raises(LivecapError):
        ctx.set_body_parts(bp, 0, 33)
    with pytest.raises(LivecapError):
        ctx.set_body_parts(np.full(23, 300, np.int32), 0, 10)
    ctx.close()
