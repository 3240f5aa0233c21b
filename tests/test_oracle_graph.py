"""Pins for the oracle's graph construction: brute force on tiny inputs."""
import math

import numpy as np
import pytest

from oracle import graph


def _rand_pts(n, seed):
    return np.random.default_rng(seed).normal(size=(n, 3)).astype(np.float32)


def _d2(a, b):
    # plain Python floats (IEEE doubles), same operation order
    dx, dy, dz = float(a[0]) - float(b[0]), float(a[1]) - float(b[1]), float(a[2]) - float(b[2])
    return (dx * dx + dy * dy) + dz * dz


@pytest.mark.parametrize("seed", [0, 1])
def test_fps_brute_force(seed):
    P = _rand_pts(60, seed)
    n = 12
    sel = [0]
    for _ in range(1, n):
        best, bj = -1.0, -1
        for j in range(len(P)):
            d = min(_d2(P[j], P[s]) for s in sel)
            if d > best:
                best, bj = d, j
        sel.append(bj)
    assert graph.farthest_point_sampling(P, n).tolist() == sel


def test_fps_ties_lowest_index():
    P = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0]], dtype=np.float32)
    assert graph.farthest_point_sampling(P, 2).tolist() == [0, 1]


@pytest.mark.parametrize("K", [1, 4])
def test_binding_brute_force(K):
    V = _rand_pts(40, 3)
    G = _rand_pts(9, 4)
    idx, w = graph.bind_vertices(V, G, K)
    for i in range(len(V)):
        keyed = sorted((_d2(V[i], G[k]), k) for k in range(len(G)))
        assert idx[i].tolist() == [k for _, k in keyed[:K]]
        dmax = math.sqrt(keyed[K][0])
        raw = [(1.0 - math.sqrt(d) / dmax) ** 2 for d, _ in keyed[:K]]
        s = sum(raw)
        ref = [r / s for r in raw] if s > 0 else [1.0 / K] * K
        assert np.allclose(w[i], ref, rtol=1e-14, atol=0)
    assert np.allclose(w.sum(1), 1.0)


def test_binding_degenerate_uniform():
    # all nodes equidistant from the vertex -> (1 - d/dmax) = 0 -> uniform
    V = np.zeros((1, 3), dtype=np.float32)
    G = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, -1, 0]], dtype=np.float32)
    idx, w = graph.bind_vertices(V, G, 4)
    assert idx.tolist() == [[0, 1, 2, 3]]
    assert np.allclose(w, 0.25)


def test_edges_brute_force_and_symmetric():
    G = _rand_pts(15, 5)
    E = graph.node_edges(G)
    ref = set()
    for k in range(len(G)):
        keyed = sorted((_d2(G[k], G[l]), l) for l in range(len(G)) if l != k)
        for _, l in keyed[:4]:
            ref.add((k, l))
            ref.add((l, k))
    assert sorted(ref) == [tuple(e) for e in E.tolist()]
    deg = np.bincount(E[:, 0], minlength=len(G))
    assert (deg >= 4).all()


def test_edge_weights_average():
    mat = np.array([1.0, 0.2, 1.0, 0.2])
    s = graph.edge_weights(mat, np.array([0, 1, 2]), np.array([[0, 1], [1, 0], [0, 2]]))
    assert np.allclose(s, [0.6, 0.6, 1.0])


def test_tiny_graph_sizes(tiny_graph, tiny_scene):
    g = tiny_graph
    assert len(g["node_vid"]) == 64 and len(set(g["node_vid"].tolist())) == 64
    assert g["bind_idx"].shape == (tiny_scene.N, 4)
    assert np.isin(np.round(g["edge_s"], 6), [0.2, 0.6, 1.0]).all()
