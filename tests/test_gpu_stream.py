"""Tracked streams: one CUDA graph per frame step over several captures
(lc_batch_step) against the same calls made one after the other.

Per member and frame the step runs the pose solve (from the explicit Euler
start or from the last solved pose), the identity start of the non-rigid
stage unless the graph parameters are carried, the warm start (with a
network), the batched non-rigid stage, the motion record and the end of the
pose frame.  The reference path makes those calls one by one (lc_pose_extrapolate,
lc_solve_pose, lc_warm_start, lc_batch_solve with from_identity = 0,
lc_record_motion, lc_pose_advance) on twin contexts: node parameters, poses
and energies must be bit-identical after every step, with and without a
network, with and without body-part masks.  Frames come from ``synth.stream_frame`` (AR(1) joint angles and
control-point field) on a small body capture.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N_STREAMS, N_FRAMES = 2, 5


@pytest.fixture(scope="module")
def capture():
    sc = synth.make_scene("body", rings=8, segments=14, side=256, n_nodes=80, frame=False)
    frames = [[synth.stream_frame(sc, 40 + j, i) for i in range(N_FRAMES)] for j in range(N_STREAMS)]
    return sc, frames


def _contexts(sc, parts=False):
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    out = []
    for _ in range(N_STREAMS):
        c = Context(0)
        setup_scene(c, sc, with_frame=False)
        c.set_params(n_gn=3, n_pcg=8)
        if parts:
            c.set_body_parts(sc.skeleton["bone_part"], sc.skeleton["torso_part"], 10)
        out.append(c)
    return out


def _first_two(ctxs, frames, net, euler=True, carry=True):
    from paper_1810_02648_gb300 import warmstart as ws
    for i in range(2):
        for j, c in enumerate(ctxs):
            ws._upload(c, frames[j][i])
            if i > 0 and euler:
                c.pose_extrapolate()
            c.solve_pose(stats=False)
            if not carry:
                c.set_node_params(None, None)
                c.record_motion()
            if i > 0 and net is not None:
                c.warm_start(net, sync=False)
            c.solve_nonrigid(stats=False)
            c.record_motion()
            c.pose_advance()


def _state(ctxs):
    out = []
    for c in ctxs:
        r = c.read_back(V=True, flags=False, pose=True)
        st = c.read_stats()
        out.append((r["R"], r["t"], r["V"], r["pose"], st["e_total"], tuple(st["e_gn"])))
    return out


@pytest.mark.parametrize("with_net,parts,euler,carry", [(False, False, True, True), (True, True, False, False),
                                                        (True, False, True, False)])
def test_step_graph_equals_the_calls(capture, with_net, parts, euler, carry):
    from paper_1810_02648_gb300 import MLP, Batch
    from paper_1810_02648_gb300 import warmstart as ws
    sc, frames = capture
    net = MLP(0, ws.init_params(5) * 0.05) if with_net else None
    ref_ctxs, step_ctxs = _contexts(sc, parts), _contexts(sc, parts)
    _first_two(ref_ctxs, frames, net, euler, carry)
    _first_two(step_ctxs, frames, net, euler, carry)
    ref_batch, step_batch = Batch(ref_ctxs), Batch(step_ctxs)
    for i in range(2, N_FRAMES):
        for j in range(N_STREAMS):
            ws._upload(ref_ctxs[j], frames[j][i])
            ws._upload(step_ctxs[j], frames[j][i])
        for c in ref_ctxs:
            if euler:
                c.pose_extrapolate()
            c.solve_pose(stats=False)
            if not carry:
                c.set_node_params(None, None)
                c.record_motion()
            if net is not None:
                c.warm_start(net, sync=False)
        ref_stats = ref_batch.solve(False, stats=True)
        for c in ref_ctxs:
            c.record_motion()
            c.pose_advance()
        step_stats = step_batch.step(net, euler_start=euler, carry_graph=carry, stats=True)
        a, b = _state(ref_ctxs), _state(step_ctxs)
        for j in range(N_STREAMS):
            for x, y in zip(a[j], b[j]):
                if isinstance(x, np.ndarray):
                    assert np.array_equal(x, y), (i, j)
                else:
                    assert x == y, (i, j)
            assert step_stats[j]["e_total"] == ref_stats[j]["e_total"]
        assert step_stats[0]["n_kernels"] > ref_stats[0]["n_kernels"]
    # the energies stay those of a tracked capture (no blow-up)
    assert all(np.isfinite(s["e_total"]) for s in step_stats)
    for bt in (ref_batch, step_batch):
        bt.close()
    for c in ref_ctxs + step_ctxs:
        c.close()
    if net is not None:
        net.close()


def test_step_needs_two_recorded_frames(capture):
    from paper_1810_02648_gb300 import Batch
    from paper_1810_02648_gb300.livecap import LC_ERR_STATE, LivecapError
    from paper_1810_02648_gb300 import warmstart as ws
    sc, frames = capture
    ctxs = _contexts(sc)
    for j, c in enumerate(ctxs):
        ws._upload(c, frames[j][0])
        c.solve_pose(stats=False)
        c.solve_nonrigid(stats=False)
        c.record_motion()
        c.pose_advance()
    batch = Batch(ctxs)
    with pytest.raises(LivecapError) as ei:
        batch.step(None)
    assert ei.value.status == LC_ERR_STATE
    batch.close()
    for c in ctxs:
        c.close()


def test_graph_warp_matches_oracle(capture):
    """The graph stage's displacement warping (lc_params.graph_warp): node
    parameters recorded in the rest pose by lc_pose_advance at one pose and
    posed by the next pose solve at its solved pose, against the oracle's
    graph_rest_params / graph_posed_params with the blend rotations of the
    two poses' bones; off, or after lc_pose_clear_history, the pose solve
    leaves the node parameters as they are."""
    from gpu_helpers import random_params, report
    from oracle import pose as opose
    from oracle import surface as osf
    from paper_1810_02648_gb300 import warmstart as ws
    sc, frames = capture
    sk = opose.skeleton_from_scene(sc)
    n = sc.n_nodes
    ctxs = _contexts(sc)
    c, off = ctxs
    c.set_params(graph_warp=1)
    R0, t0 = random_params(n, 77, rot=0.2, trans=0.02)
    for ctx in (c, off):
        ws._upload(ctx, frames[0][0])
        ctx.solve_pose(stats=False)
        ctx.set_node_params(R0.reshape(n, 9), t0)
        ctx.pose_advance()
    p1 = c.read_back(V=False, flags=False, pose=True)
    for ctx in (c, off):
        ws._upload(ctx, frames[0][3])
        ctx.solve_pose(stats=False)
    p2 = c.read_back(V=False, flags=False, pose=True)
    node_vid = c.read_graph()["node_vid"]

    def Q_of(pose):
        G, _ = opose.forward_kinematics(sk, *opose.split_pose(sk, pose))
        return osf.blend_rotations(G, sc.skeleton["skin_idx"], sc.skeleton["skin_w"])

    Rr, tr = osf.graph_rest_params(p1["R"], p1["t"], node_vid, Q_of(p1["pose"]))
    R2, t2 = osf.graph_posed_params(Rr, tr, node_vid, Q_of(p2["pose"]))
    dR = np.abs(p2["R"].reshape(n, 3, 3) - R2).max()
    dt = np.abs(p2["t"] - t2).max()
    moved = np.abs(R2 - p1["R"].reshape(n, 3, 3)).max()
    report("graph_warp", dR=dR, dt=dt, rotation_change=moved)
    assert moved > 1e-3                      # the pose change did rotate the parameters
    assert dR <= 1e-5 and dt <= 1e-6
    q = off.read_back(V=False, flags=False)
    assert np.array_equal(q["R"].reshape(n, 9), R0.reshape(n, 9)) and np.array_equal(q["t"], t0)
    # a cleared history drops the record
    c.pose_clear_history()
    before = c.read_back(V=False, flags=False)
    c.solve_pose(stats=False)
    after = c.read_back(V=False, flags=False)
    assert np.array_equal(before["R"], after["R"]) and np.array_equal(before["t"], after["t"])
    for ctx in ctxs:
        ctx.close()
