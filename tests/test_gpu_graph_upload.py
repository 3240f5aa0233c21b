"""A caller-built embedded graph (lc_upload_graph) against the library's own
build and the FP64 oracle.

* The library's graph read back and uploaded into a second context gives a
  bit-identical solve.
* A graph built outside the library by the oracle's routines, with another
  structure (random node vertices, K = 3, six-nearest node edges, uniform
  ARAP weights), solves on the GPU within the end-to-end tolerances of the
  built graph: final energy within 1e-4 (relative) of the oracle's on the
  same graph, every step's energy too, vertices within 1e-4 of the
  template's bounding-box diagonal.
* Malformed graphs are rejected with LC_ERR_ARG on the host, leaving the
  previous graph in place; a valid upload on the same context then works.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import graph_from_gpu, report
from oracle import graph as ograph
from oracle import nonrigid as onr

pytestmark = pytest.mark.gpu


def _ctx(scene, **params):
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    ctx = Context(0)
    setup_scene(ctx, scene)
    if params:
        ctx.set_params(**params)
    return ctx


def _csr(n, edges, s):
    """Directed edge list (E x 2) and weights -> CSR by source node."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    order = np.lexsort((edges[:, 1], edges[:, 0]))
    e = edges[order]
    off = np.searchsorted(e[:, 0], np.arange(n + 1)).astype(np.int32)
    return off, e[:, 1].astype(np.int32), np.asarray(s, dtype=np.float32)[order]


def _upload(ctx, g):
    n = len(g["node_vid"])
    off, dst, es = _csr(n, g["edges"], g["edge_s"])
    ctx.upload_graph(g["node_vid"], g["bind_idx"], g["bind_w"], off, dst, es)


@pytest.fixture(scope="module")
def tiny():
    return synth.make_scene("tiny")


def test_uploaded_copy_of_built_graph_solves_identically(tiny):
    a = _ctx(tiny)
    sa = a.solve_nonrigid()
    ga = a.read_graph()
    b = _ctx(tiny)
    b.upload_graph(ga["node_vid"], ga["bind_idx"], ga["bind_w"], ga["edge_off"], ga["edge_dst"], ga["edge_s"])
    gb = b.read_graph()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    sb = b.solve_nonrigid()
    assert sb["e_total"] == sa["e_total"] and sb["e_gn"] == sa["e_gn"]
    assert np.array_equal(a.read_back()["V"], b.read_back()["V"])
    a.close()
    b.close()


def _custom_graph(scene, n_nodes=48, K=3, seed=7):
    rng = np.random.default_rng(seed)
    V32 = scene.V.astype(np.float32)
    vid = np.sort(rng.choice(len(V32), size=n_nodes, replace=False)).astype(np.int64)
    G32 = V32[vid]
    idx, w = ograph.bind_vertices(V32, G32, K)
    edges = ograph.node_edges(G32, k_edges=6)
    s = np.full(len(edges), 0.7)
    return dict(node_vid=vid, bind_idx=idx, bind_w=w.astype(np.float32).astype(np.float64), edges=edges, edge_s=s)


@pytest.mark.parametrize("n_pcg", [3, None])
def test_caller_graph_matches_oracle(tiny, n_pcg):
    g = _custom_graph(tiny)
    ctx = _ctx(tiny)
    if n_pcg is not None:
        ctx.set_params(n_pcg=n_pcg)
    _upload(ctx, g)
    rb = ctx.read_graph()
    assert np.array_equal(rb["node_vid"], g["node_vid"]) and np.array_equal(rb["bind_idx"], g["bind_idx"])
    assert ctx.K == 3 and ctx.n == 48
    st = ctx.solve_nonrigid()
    out = ctx.read_back()
    graph = graph_from_gpu(rb)
    ref = onr.solve_scene(tiny, graph=graph, n_pcg=n_pcg)
    e_gpu, e_ref = st["e_total"], ref["e1"]["total"]
    rel = abs(e_gpu - e_ref) / abs(e_ref)
    diag = np.linalg.norm(tiny.V.max(0) - tiny.V.min(0))
    dv = np.abs(out["V"].astype(np.float64) - ref["v"]).max()
    hist = np.array(st["e_gn"])
    hist_ref = np.array([h["energy"] for h in ref["hist"]])
    report(f"upload_graph_e2e_{n_pcg}", e_gpu=e_gpu, e_ref=e_ref, rel=rel, dv_over_diag=dv / diag,
           hist_rel=(np.abs(hist - hist_ref) / hist_ref).max(), e_start=ref["e0"]["total"])
    assert e_gpu < ref["e0"]["total"]            # the solve made progress on this graph
    assert rel <= 1e-4
    assert dv <= 1e-4 * diag
    assert (np.abs(hist - hist_ref) <= 1e-4 * hist_ref).all()
    ctx.close()


def test_malformed_graphs_are_rejected(tiny):
    from paper_1810_02648_gb300.livecap import LC_ERR_ARG, LivecapError
    ctx = _ctx(tiny)
    ga = ctx.read_graph()
    before = ctx.solve_nonrigid()["e_total"]
    n = len(ga["node_vid"])
    base = dict(node_vid=ga["node_vid"], bind_idx=ga["bind_idx"], bind_w=ga["bind_w"], edge_off=ga["edge_off"],
                edge_dst=ga["edge_dst"], edge_s=ga["edge_s"])

    def bad(**over):
        args = dict(base)
        args.update(over)
        with pytest.raises(LivecapError) as ei:
            ctx.upload_graph(**args)
        assert ei.value.status == LC_ERR_ARG

    vid = ga["node_vid"].copy(); vid[3] = tiny.N
    bad(node_vid=vid)
    bi = ga["bind_idx"].copy(); bi[10, 1] = n
    bad(bind_idx=bi)
    bw = ga["bind_w"].copy(); bw[5, 0] = -0.1
    bad(bind_w=bw)
    bw = ga["bind_w"].copy(); bw[5, 0] = np.nan
    bad(bind_w=bw)
    es = ga["edge_s"].copy(); es[0] *= 2.0                       # unequal weights of a pair
    bad(edge_s=es)
    ed = ga["edge_dst"].copy(); ed[0] = 0                        # node 0's first edge to itself
    bad(edge_dst=ed)
    ed = ga["edge_dst"].copy()
    k0 = int(np.searchsorted(ga["edge_off"], 0, side="right") - 1)
    ed[0] = (ed[0] + 1) % n if (ed[0] + 1) % n != k0 else (ed[0] + 2) % n    # reverse edge missing
    bad(edge_dst=ed)
    off = ga["edge_off"].copy(); off[2], off[3] = off[3], off[2]
    bad(edge_off=off)
    off = ga["edge_off"].copy(); off[0] = 1
    bad(edge_off=off)
    # the previous graph is still in place, and a valid upload works after the failures
    ctx.set_node_params(None, None)
    assert ctx.solve_nonrigid()["e_total"] == before
    ctx.upload_graph(**base)
    ctx.set_node_params(None, None)
    assert ctx.solve_nonrigid()["e_total"] == before
    ctx.close()


def test_graph_without_edges(tiny):
    """No ARAP edges: the data terms alone, against the oracle at three
    PCG iterations."""
    g = _custom_graph(tiny)
    g = dict(g, edges=np.zeros((0, 2), np.int64), edge_s=np.zeros(0))
    ctx = _ctx(tiny, n_pcg=3, n_gn=2)
    _upload(ctx, g)
    st = ctx.solve_nonrigid()
    rb = ctx.read_graph()
    assert len(rb["edge_dst"]) == 0
    ref = onr.solve_scene(tiny, graph=graph_from_gpu(rb), n_pcg=3, n_gn=2)
    rel = abs(st["e_total"] - ref["e1"]["total"]) / ref["e1"]["total"]
    report("upload_graph_no_edges", rel=rel)
    assert rel <= 1e-4
    ctx.close()
