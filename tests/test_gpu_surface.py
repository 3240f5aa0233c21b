"""GPU parity of the per-vertex surface stage against the FP64 oracle
(oracle/surface.py), through the C ABI.

* frame decisions at the surface (z-buffer keys, visibility, contour set,
  b_i, projections): bit-exact;
* at identical FP32 vertex positions: the six energies within 1e-5
  (relative; FP32 sums inside a tile, FP64 across tiles), -J^T F,
  diag(J^T J) and J^T J p within 1e-4 of the vector's largest entry (FP32
  accumulation over a vertex's data block and one-ring);
* PCG: identical iteration counts, the quadratic model within 1e-4, the
  iterate within max(1e-4, twice the spread of FP32 executions of the same
  CG measured on the oracle's matrix);
* end to end (3 Gauss-Newton x 4 PCG, Sec. 4): final energy and vertices
  within max(strict bound, twice the oracle's own spread under FP32
  rounding), strict bound 1e-4 relative energy and 1e-4 x the bounding-box
  diagonal;
* displacement warping against the oracle's blended rotations at the
  kinematics of the GPU's pose.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import _r32, pcg32, ragged_scene, report, surface_rounding_band
from oracle import nonrigid as onr
from oracle import pose as opose
from oracle import surface as osf
from oracle import visibility as ovis

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


def _start(scene, kind, seed=0):
    """(FP32 start surface, FP32 rest geometry V^S or None for the template).
    V^S: the template, or for a body scene its ground-truth pose without the
    non-rigid part (synthetic, in place of a pose stage's skinned mesh); the
    start is V^S plus a smooth seeded offset."""
    VS = np.asarray(scene.meta["V_posed"] if kind == "posed" else scene.V, dtype=np.float32)
    V = VS.astype(np.float64)
    rng = np.random.default_rng(seed)
    c = V.mean(0)
    off = 0.004 * np.sin((V - c) @ rng.normal(size=(3, 3)) * 6.0)
    return (V + off).astype(np.float32), (VS if kind == "posed" else None)


def _oracle_flags(P, flags):
    P.vis = (flags & ovis.FLAG_VISIBLE) != 0
    P.inB = (flags & ovis.FLAG_INB) != 0
    P.bsign = np.where((flags & ovis.FLAG_BNEG) != 0, -1.0, 1.0)


def _cases(tiny, body):
    return {"tiny": (tiny, "template"), "body": (body, "posed")}


# ---------------------------------------------------------------------------
# frame decisions at the surface: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["tiny", "body", "ragged"])
def test_surface_visibility_bit_exact(case, tiny, body):
    scene, kind = _cases(tiny, body).get(case, (None, "template"))
    if case == "ragged":
        scene = ragged_scene(20, 16, 40, 4, side=80, shift=0.45)
    V0, _ = _start(scene, kind, 1)
    ctx = _ctx(scene)
    ctx.set_surface(V0)
    ctx.surface_visibility()
    vis = ctx.read_visibility()
    ref = ovis.visibility(V0, scene.F, scene.cam.f, scene.cam.cx, scene.cam.cy, scene.cam.W, scene.cam.H,
                          scene.dt, scene.mask.astype(np.uint8))
    assert np.array_equal(vis["uv"], ref["uv"])
    assert np.array_equal(vis["zbuf"], ref["zbuf"])
    assert np.array_equal(vis["flags"], ref["flags"])
    V, flags = ctx.read_surface(flags=True)
    assert np.array_equal(V, V0) and np.array_equal(flags, ref["flags"])
    report(f"surface_vis_{case}", n_vis=int((ref["flags"] & 1).astype(bool).sum()),
           n_B=int(((ref["flags"] & 4) != 0).sum()))
    ctx.close()


# ---------------------------------------------------------------------------
# linearisation, J^T J p and PCG at identical FP32 positions
# ---------------------------------------------------------------------------
def _lin_case(scene, kind, tag, history=False, collapse=False, seed=2):
    V0, VS = _start(scene, kind, seed)
    if collapse:
        # two neighbours on the same point: a zero-length edge (zero E_edge row)
        off, dst = osf.one_ring(len(V0), scene.F)
        V0[dst[off[7]]] = V0[7]
    ctx = _ctx(scene)
    prev1 = prev2 = None
    if history:
        rng = np.random.default_rng(seed + 1)
        prev1 = (V0 + rng.normal(scale=0.003, size=V0.shape)).astype(np.float32)
        prev2 = (V0 + rng.normal(scale=0.003, size=V0.shape)).astype(np.float32)
        ctx.surface_history(prev1, prev2)
    if VS is not None:
        ctx.set_rest_geometry(VS)
    ctx.set_surface(V0)
    ctx.surface_visibility()
    flags = ctx.read_visibility()["flags"]
    lin = ctx.surface_linearize()
    P = osf.problem_from_scene(scene, base32=VS, prev1=prev1, prev2=prev2)
    _oracle_flags(P, flags)
    V = V0.astype(np.float64)
    e_ref = osf.energy(P, V)
    e_vec = np.array([e_ref[k] for k in ("photo", "sil", "smooth", "edge", "velocity", "acceleration")])
    d_en = np.abs(lin["energy"] - e_vec) / np.maximum(np.abs(e_vec), 1e-12)
    A, b, F, J = osf.normal_equations(P, V)
    JT = J.T.tocsr()
    diag_ref = np.asarray(JT.multiply(JT).sum(1)).ravel()
    d_rhs = np.abs(lin["rhs"].ravel() - b).max() / np.abs(b).max()
    d_diag = np.abs(lin["diag"].ravel() - diag_ref).max() / np.abs(diag_ref).max()
    rng = np.random.default_rng(seed + 2)
    p = rng.normal(size=V.shape).astype(np.float32)
    Ap = ctx.surface_apply_jtj(p)
    Ap_ref = A @ p.astype(np.float64).ravel()
    d_Ap = np.abs(Ap.ravel() - Ap_ref).max() / np.abs(Ap_ref).max()
    report(f"surface_lin_{tag}", energy=d_en.max(), rhs=d_rhs, diag=d_diag, jtjp=d_Ap,
           n_vis=int(P.vis.sum()), n_B=int(P.inB.sum()))
    assert d_en.max() <= 1e-5
    assert d_rhs <= 1e-4 and d_diag <= 1e-4 and d_Ap <= 1e-4
    if not history:
        assert lin["energy"][4] == 0.0 and lin["energy"][5] == 0.0

    q = lambda d: 0.5 * d @ (A @ d) - b @ d  # noqa: E731
    for n_pcg in (1, 4, 12):
        ctx.set_params(n_pcg_surface=n_pcg)
        delta, iters = ctx.surface_solve_linear()
        dref, info = onr.pcg(A, b, n_pcg)
        band = 0.0
        for s in range(3):
            d32, _ = pcg32(A, b, n_pcg, _r32(np.random.default_rng(4000 + s)))
            band = max(band, np.linalg.norm(d32 - dref) / np.linalg.norm(dref))
        d_pcg = np.linalg.norm(delta.ravel() - dref) / np.linalg.norm(dref)
        d_q = abs(q(delta.ravel().astype(np.float64)) - q(dref)) / abs(q(dref))
        report(f"surface_pcg_{tag}_{n_pcg}", rel=d_pcg, band=band, q_rel=d_q, iters=iters)
        assert iters == info["iters"]
        assert d_pcg <= max(1e-4, 2.0 * band) and d_q <= 1e-4
    ctx.close()


@pytest.mark.parametrize("history", [False, True])
def test_surface_linearization_tiny(tiny, history):
    _lin_case(tiny, "template", f"tiny_h{int(history)}", history=history)


@pytest.mark.parametrize("history", [False, True])
def test_surface_linearization_body(body, history):
    _lin_case(body, "posed", f"body_h{int(history)}", history=history)


def test_surface_linearization_ragged():
    _lin_case(ragged_scene(13, 11, 37, 3, side=70, shift=0.3), "template", "ragged", history=True)


def test_surface_linearization_zero_length_edge(tiny):
    _lin_case(tiny, "template", "collapsed", collapse=True)


# ---------------------------------------------------------------------------
# end to end
# ---------------------------------------------------------------------------
def _e2e(scene, kind, tag, history=False, seed=3, pcg_kernel=0):
    V0, VS = _start(scene, kind, seed)
    ctx = _ctx(scene, pcg_kernel=pcg_kernel)
    if VS is not None:
        ctx.set_rest_geometry(VS)
    prev1 = prev2 = None
    if history:
        rng = np.random.default_rng(seed + 1)
        prev1 = (V0 + rng.normal(scale=0.002, size=V0.shape)).astype(np.float32)
        prev2 = (V0 + rng.normal(scale=0.002, size=V0.shape)).astype(np.float32)
        ctx.surface_history(prev1, prev2)
    ctx.set_surface(V0)
    stats = ctx.solve_surface()
    V, flags = ctx.read_surface(flags=True)
    ref, band_E, band_V = surface_rounding_band(scene, base32=VS, V0=V0, prev1=prev1, prev2=prev2)
    P = ref["problem"]
    e_gpu, e_ref = stats["e_total"], ref["e1"]["total"]
    rel = abs(e_gpu - e_ref) / abs(e_ref)
    diag = np.linalg.norm(scene.V.max(0) - scene.V.min(0))
    dv = np.abs(V.astype(np.float64) - ref["V"]).max()
    e_hist = np.array(stats["e_gn"])
    e_hist_ref = np.array([h["energy"] for h in ref["hist"]])
    report(f"surface_e2e_{tag}", e_gpu=e_gpu, e_ref=e_ref, rel=rel, dv=dv, dv_over_diag=dv / diag,
           band_E_rel=band_E / abs(e_ref), band_V=band_V,
           hist_rel=np.abs(e_hist - e_hist_ref).max() / e_hist_ref.max(), n_kernels=stats["n_kernels"],
           e0=ref["e0"]["total"])
    assert stats["pcg_iters"] == [h["pcg_iters"] for h in ref["hist"]]
    assert np.array_equal((flags & ovis.FLAG_VISIBLE) != 0, P.vis)
    assert np.array_equal((flags & ovis.FLAG_INB) != 0, P.inB)
    assert stats["n_visible"] == int(P.vis.sum()) and stats["n_boundary"] == int(P.inB.sum())
    assert abs(e_gpu - e_ref) <= max(1e-4 * abs(e_ref), 2.0 * band_E)
    assert dv <= max(1e-4 * diag, 2.0 * band_V)
    assert np.abs(e_hist - e_hist_ref).max() <= max(1e-4 * e_hist_ref.max(), 2.0 * band_E)
    for k, key in (("e_smooth", "smooth"), ("e_edge", "edge"), ("e_velocity", "velocity"),
                   ("e_acceleration", "acceleration")):
        assert abs(stats[k] - ref["e1"][key]) <= max(1e-4 * abs(e_ref), 2.0 * band_E)
    assert stats["e_arap"] == 0.0
    # the solve lowers the energy, and replaying it from the same start is bit-identical
    assert e_gpu < ref["e0"]["total"]
    ctx.set_surface(V0)
    stats2 = ctx.solve_surface()
    assert stats2["e_total"] == e_gpu and np.array_equal(ctx.read_surface(), V)
    assert ctx.read_stats()["e_total"] == e_gpu
    ctx.close()
    return stats


def test_surface_end_to_end_tiny(tiny):
    _e2e(tiny, "template", "tiny")


@pytest.mark.parametrize("history", [False, True])
def test_surface_end_to_end_body(body, history):
    st = _e2e(body, "posed", f"body_h{int(history)}", history=history)
    assert 1 <= st["pcg_cluster_size"] <= 16


@pytest.mark.parametrize("case", ["tiny", "body"])
def test_surface_pcg_paths_bit_identical(case, tiny, body):
    """The cluster-persistent PCG (default for captures of <= 64 vertex
    tiles) reduces every dot product per tile in the order of the
    per-iteration kernels (pcg_kernel 1): both solves give identical bits."""
    scene, kind = _cases(tiny, body)[case]
    V0, VS = _start(scene, kind, 5)
    out = []
    for k in (0, 1):
        ctx = _ctx(scene, pcg_kernel=k)
        if VS is not None:
            ctx.set_rest_geometry(VS)
        ctx.set_surface(V0)
        st = ctx.solve_surface()
        out.append((st, ctx.read_surface()))
        ctx.close()
    (s0, v0), (s1, v1) = out
    assert 1 <= s0["pcg_cluster_size"] <= 16 and s1["pcg_cluster_size"] == 0
    assert np.array_equal(v0, v1)
    assert s0["e_total"] == s1["e_total"] and s0["e_gn"] == s1["e_gn"] and s0["pcg_iters"] == s1["pcg_iters"]


def test_surface_end_to_end_ragged():
    _e2e(ragged_scene(15, 13, 41, 4, side=90, shift=0.2), "template", "ragged", history=True)


def test_surface_empty_frame():
    s = synth.make_scene("tiny")
    s.rgb = np.zeros_like(s.rgb)
    s.dt = np.zeros_like(s.dt)
    s.mask = np.zeros_like(s.mask)
    st = _e2e(s, "template", "empty")
    assert st["n_boundary_neg"] == 0


def test_surface_target_energy_stop(tiny):
    """A target above the start energy: no update is made."""
    V0, _ = _start(tiny, "template", 4)
    ctx = _ctx(tiny)
    ctx.set_surface(V0)
    st = ctx.solve_surface()
    ctx.set_params(target_energy=float(st["e_gn"][0]) * 2.0)
    ctx.set_surface(V0)
    st2 = ctx.solve_surface()
    assert st2["n_gn_done"] == 0
    assert np.array_equal(ctx.read_surface(), V0)
    ctx.close()


# ---------------------------------------------------------------------------
# history and displacement warping
# ---------------------------------------------------------------------------
def _oracle_Q(scene, pose):
    sk = opose.skeleton_from_scene(scene)
    R_root, t_root, ang = opose.split_pose(sk, pose.astype(np.float64))
    G, o = opose.forward_kinematics(sk, R_root, t_root, ang)
    return osf.blend_rotations(G, scene.skeleton["skin_idx"], scene.skeleton["skin_w"])


def test_surface_advance_and_displacement_warping(body):
    ctx = _ctx(body, n_gn_pose=2)
    # frame a: pose stage, then a displaced surface, then advance
    ctx.solve_pose(stats=False)
    pose_a = ctx.read_back(R=False, t=False, V=False, flags=False, pose=True)["pose"]
    VS_a = ctx.eval_pose()["V"]
    rng = np.random.default_rng(6)
    d = (0.005 * rng.normal(size=VS_a.shape)).astype(np.float32)
    Va = (VS_a + d).astype(np.float32)
    ctx.set_surface(Va)
    ctx.surface_advance()
    # same pose: the start returns the surface (FP32 rotation round trip)
    ctx.surface_start()
    back = ctx.read_surface()
    assert np.abs(back - Va).max() <= 4e-7 * np.abs(Va).max() + 1e-6 * np.abs(d).max()
    # frame b from another start pose: V = V^S_b + Q_b Q_a^T (Va - V^S_a)
    pose_b0 = body.pose_init.copy()
    pose_b0[6:] += 0.1
    ctx.set_pose(pose_b0)
    ctx.solve_pose(stats=False)
    pose_b = ctx.read_back(R=False, t=False, V=False, flags=False, pose=True)["pose"]
    VS_b = ctx.eval_pose()["V"]
    ctx.surface_start()
    Vb = ctx.read_surface()
    Qa, Qb = _oracle_Q(body, pose_a), _oracle_Q(body, pose_b)
    dh = osf.record_displacement(Va, VS_a, Qa)
    ref = osf.warped_start(VS_b, Qb, dh)
    err = np.abs(Vb - ref).max()
    report("surface_warp_body", err=err, max_rot_change=float(np.abs(Qb - Qa).max()))
    assert np.abs(Qb - Qa).max() > 1e-2          # the poses differ enough to matter
    assert err <= 2e-6 + 1e-4 * np.abs(d).max()
    # the history holds V_a: a second advance shifts it to V^{t-2}
    ctx.set_surface(Vb)
    ctx.surface_advance()
    P = osf.problem_from_scene(body, base32=VS_b, prev1=Vb, prev2=Va)
    ctx.surface_visibility()
    _oracle_flags(P, ctx.read_visibility()["flags"])
    lin = ctx.surface_linearize()
    e = osf.energy(P, Vb.astype(np.float64))
    assert lin["energy"][4] == 0.0                               # V = V^{t-1}
    assert abs(lin["energy"][5] - e["acceleration"]) <= 1e-5 * e["acceleration"]
    ctx.close()


def test_surface_without_skeleton_start(tiny):
    """Without a skeleton the warp is the identity: start = V^S + (V - V^S)."""
    ctx = _ctx(tiny)
    V0, _ = _start(tiny, "template", 7)
    ctx.surface_start()
    assert np.array_equal(ctx.read_surface(), tiny.V)          # no displacement yet: V^S
    ctx.set_surface(V0)
    ctx.surface_advance()
    ctx.surface_start()
    assert np.abs(ctx.read_surface() - V0).max() <= 1e-6
    ctx.close()
