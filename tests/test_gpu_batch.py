"""Batched captures (lc_batch_*): uneven meshes, node counts, K and images
solved together in one launch per phase.

Each capture keeps its own buffers and reductions, so under the same PCG
strategy its batched result must equal its own single-context solve bit for
bit (node parameters, vertices, flags, energies, iteration counts).  That,
plus the single-context parity against the oracle, carries the oracle parity
over to the batch; one member is also compared with the oracle directly.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import graph_from_gpu, ragged_scene, report

pytestmark = pytest.mark.gpu

N_GN, N_PCG = 3, 10


def _scenes():
    out = [synth.make_scene("tiny"),
           ragged_scene(13, 11, 37, 3),                   # K = 3, odd image
           ragged_scene(17, 9, 50, 8, side=80, shift=0.45),   # K = 8, leaves the image
           ragged_scene(6, 7, 5, 4)]                      # 5 nodes: too few for a cluster
    out += synth.make_batch(count=3, seed=7, n_min=2000, n_max=4000, side_min=256, side_max=384)
    return out


@pytest.fixture(scope="module")
def scenes():
    return _scenes()


def _contexts(scenes, pcg_kernel):
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    ctxs = []
    for sc in scenes:
        c = Context(0)
        setup_scene(c, sc)
        c.set_params(n_gn=N_GN, n_pcg=N_PCG, pcg_kernel=pcg_kernel)
        ctxs.append(c)
    return ctxs


def _single(ctxs):
    res = []
    for c in ctxs:
        c.set_node_params(None, None)
        st = c.solve_nonrigid()
        res.append((st, c.read_back()))
    return res


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("R", "t", "V", "flags"))


@pytest.mark.parametrize("mode,pcg_kernel", [(0, 0), (3, 1)])
def test_batch_equals_single_solves(scenes, mode, pcg_kernel):
    from paper_1810_02648_gb300 import Batch
    ctxs = _contexts(scenes, pcg_kernel)
    ref = _single(ctxs)
    b = Batch(ctxs)
    b.set_pcg_mode(mode)
    stats = b.solve(from_identity=True)
    clusters = []
    for i, c in enumerate(ctxs):
        out = c.read_back()
        st_ref, out_ref = ref[i]
        assert _same(out, out_ref), f"capture {i}"
        assert stats[i]["e_total"] == st_ref["e_total"]
        assert stats[i]["e_gn"] == st_ref["e_gn"] and stats[i]["pcg_iters"] == st_ref["pcg_iters"]
        assert stats[i]["n_visible"] == st_ref["n_visible"] and stats[i]["n_boundary"] == st_ref["n_boundary"]
        assert stats[i]["pcg_cluster_size"] == st_ref["pcg_cluster_size"]
        clusters.append(stats[i]["pcg_cluster_size"])
    if mode == 0:
        assert any(clusters) and not all(clusters)   # both PCG paths in one batch
    # a second solve from the identity repeats the first exactly
    b.solve(from_identity=True, stats=False)
    for i, c in enumerate(ctxs):
        assert _same(c.read_back(), ref[i][1])
    report(f"batch_mode{mode}", captures=len(ctxs), cluster_sizes=clusters, kernels=stats[0]["n_kernels"])
    b.close()
    for c in ctxs:
        c.close()


def test_batch_member_matches_oracle(scenes):
    """One batch member (3 PCG iterations, outside CG's FP32-sensitive regime)
    against the oracle to the strict bound."""
    from paper_1810_02648_gb300 import Batch
    from oracle import nonrigid as onr
    ctxs = _contexts(scenes[:3], 0)
    for c in ctxs:
        c.set_params(n_pcg=3)
    b = Batch(ctxs)
    stats = b.solve(from_identity=True)
    sc, c = scenes[1], ctxs[1]
    ref = onr.solve_scene(sc, graph=graph_from_gpu(c.read_graph()), n_gn=N_GN, n_pcg=3)
    out = c.read_back()
    rel = abs(stats[1]["e_total"] - ref["e1"]["total"]) / ref["e1"]["total"]
    diag = np.linalg.norm(sc.V.max(0) - sc.V.min(0))
    dv = np.abs(out["V"] - ref["v"]).max()
    report("batch_member_oracle", rel=rel, dv_over_diag=dv / diag)
    assert rel <= 1e-4 and dv <= 1e-4 * diag
    b.close()
    for c in ctxs:
        c.close()


def test_batch_autotune_and_errors(scenes):
    from paper_1810_02648_gb300 import Batch, Context, LivecapError
    ctxs = _contexts(scenes[:4], 0)
    b = Batch(ctxs)
    mode, ms = b.autotune(reps=2)
    assert mode in (0, 1, 2, 3) and np.all(ms > 0)
    assert ms[mode] == ms.min()
    stats = b.solve(from_identity=True)
    assert all(np.isfinite(s["e_total"]) for s in stats)
    report("batch_autotune", mode=mode, ms=[float(x) for x in ms])
    with pytest.raises(LivecapError):
        b.set_pcg_mode(7)
    b.close()
    # members must agree in n_gn / n_pcg, and be set up
    ctxs[1].set_params(n_pcg=N_PCG + 1)
    with pytest.raises(LivecapError):
        Batch(ctxs)
    bare = Context(0)
    with pytest.raises(LivecapError):
        Batch([ctxs[0], bare])
    bare.close()
    for c in ctxs:
        c.close()


def test_batch_members_with_body_part_masks():
    """Members with a body-part mask (body captures with a skeleton) beside
    one without: each batched result equals its own single solve, and the
    masked members' silhouette rows were masked."""
    from paper_1810_02648_gb300 import Batch, Context
    from synth import setup_scene
    scs = [synth.make_scene("body", seed=s, rings=8, segments=14, side=256, n_nodes=80) for s in (3, 4)]
    scs.append(synth.make_scene("tiny"))
    ctxs = []
    for k, sc in enumerate(scs):
        c = Context(0)
        setup_scene(c, sc)
        c.set_params(n_gn=N_GN, n_pcg=N_PCG)
        if sc.skeleton is not None:
            c.solve_pose(stats=False)
            c.set_body_parts(sc.skeleton["bone_part"], sc.skeleton["torso_part"], 10)
        ctxs.append(c)
    ref = _single(ctxs)
    b = Batch(ctxs)
    stats = b.solve(from_identity=True)
    for i, c in enumerate(ctxs):
        out = c.read_back()
        st_ref, out_ref = ref[i]
        assert _same(out, out_ref), f"capture {i}"
        assert stats[i]["e_total"] == st_ref["e_total"] and stats[i]["e_gn"] == st_ref["e_gn"]
    masked = [int(((ref[i][1]["flags"] & 32) != 0).sum()) for i in range(2)]
    report("batch_body_parts", masked=masked, e=[s["e_total"] for s in stats])
    b.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("shape", [(128, 8, 2), (512, 16, 8), (256, 16, 4), (128, 16, 2)])
def test_jtj_launch_shapes_are_bit_identical(scenes, shape):
    """The per-iteration J^T J p at another launch shape (vertex block,
    warps of four nodes per node block, entry rounds in flight) gives the same bits as the
    default shape: node parameters, vertices, flags, energies."""
    from paper_1810_02648_gb300 import Batch
    from paper_1810_02648_gb300.livecap import BATCH_PCG_PER_ITERATION
    ctxs = _contexts(scenes, 1)
    b = Batch(ctxs)
    b.set_shape(BATCH_PCG_PER_ITERATION)
    ref_stats = b.solve(from_identity=True)
    ref = [c.read_back() for c in ctxs]
    vb, nw, nu = shape
    b.set_shape(BATCH_PCG_PER_ITERATION, vb, nw, nu)
    assert b.shape() == dict(pcg_mode=BATCH_PCG_PER_ITERATION, vert_block=vb, node_warps=nw, node_unroll=nu)
    stats = b.solve(from_identity=True)
    for i, c in enumerate(ctxs):
        assert _same(c.read_back(), ref[i]), f"capture {i}"
        assert stats[i]["e_gn"] == ref_stats[i]["e_gn"] and stats[i]["e_total"] == ref_stats[i]["e_total"]
        assert stats[i]["pcg_iters"] == ref_stats[i]["pcg_iters"]
    b.close()
    for c in ctxs:
        c.close()


def test_shape_autotuner_and_its_table(scenes):
    """The autotuner tries every shape of the strategies that use the
    per-iteration product, rejects none (all bit-identical), sets the
    fastest, stores it under the batch's size class, and a second batch of
    the same class takes it from the table without timing."""
    from paper_1810_02648_gb300 import Batch
    from paper_1810_02648_gb300.livecap import autotune_table
    ctxs = _contexts(scenes, 0)
    b = Batch(ctxs)
    r = b.autotune_shapes(reps=1, use_cache=False)
    report("shape_autotune", tried=r["tried"], rejected=r["rejected"], ms=r["ms"], **r["shape"])
    assert r["tried"] > 4 and r["rejected"] == 0 and not r["from_cache"]
    assert b.shape() == r["shape"]
    key = b.size_class()
    table = autotune_table()
    assert any(line.split("\t")[0] == key for line in table.splitlines())
    b2 = Batch(ctxs)
    r2 = b2.autotune_shapes(reps=1, use_cache=True)
    assert r2["from_cache"] and r2["shape"] == r["shape"] and r2["tried"] == 0
    for bt in (b, b2):
        bt.close()
    for c in ctxs:
        c.close()
