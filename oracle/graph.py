"""Embedded deformation graph construction (FP64).  TEST INFRASTRUCTURE ONLY.

The paper solves per-vertex displacements (Sec. 3.4, Discussion); the
embedded-graph form built here is the one the non-rigid solver targets: nodes
by farthest-point sampling, each vertex bound to its K nearest nodes with
weights (1 - d/d_max)^2 normalised, and node edges among nearby nodes.  Edge
weights average the two endpoints' material weights, as the paper does for
its per-edge non-rigidity weights s_ij (Sec. 3.1, Tab. 1).

Readings (the paper is silent on all of them):
* FPS starts at vertex 0; squared distances are FP64 values computed from the
  FP32 coordinates as (dx*dx + dy*dy) + dz*dz; ties go to the lowest index.
* K-nearest nodes: order by (squared distance, node index); d_max is the
  distance to the (K+1)-th nearest node; if the K weights sum to zero (or
  d_max is zero) the weights are uniform 1/K.
* Node edges: l is a neighbour of k if l is among the 4 nearest other nodes
  of k, or k among those of l.  Both directions are kept, sorted by (k, l).
"""
from __future__ import annotations

import numpy as np


def _sqdist(P: np.ndarray, q: np.ndarray) -> np.ndarray:
    """FP64 squared distances from rows of P to point q, fixed op order."""
    dx = P[:, 0] - q[0]
    dy = P[:, 1] - q[1]
    dz = P[:, 2] - q[2]
    return (dx * dx + dy * dy) + dz * dz


def farthest_point_sampling(V32: np.ndarray, n: int) -> np.ndarray:
    """Indices of n vertices: vertex 0, then repeatedly the vertex whose
    distance to the already chosen set is largest (lowest index on ties)."""
    V = np.asarray(V32, dtype=np.float32).astype(np.float64)
    if not (1 <= n <= len(V)):
        raise ValueError("need 1 <= n_nodes <= n_vertices")
    sel = [0]
    d = _sqdist(V, V[0])
    for _ in range(1, n):
        j = int(np.argmax(d))          # first maximum -> lowest index
        sel.append(j)
        d = np.minimum(d, _sqdist(V, V[j]))
    return np.asarray(sel, dtype=np.int64)


def bind_vertices(V32: np.ndarray, G32: np.ndarray, K: int):
    """K nearest nodes per vertex and their normalised weights.

    Returns (idx (N,K) int64, w (N,K) float64).  Requires n_nodes >= K+1.
    """
    V = np.asarray(V32, dtype=np.float32).astype(np.float64)
    G = np.asarray(G32, dtype=np.float32).astype(np.float64)
    n = len(G)
    if n < K + 1:
        raise ValueError("binding needs at least K+1 nodes")
    idx = np.empty((len(V), K), dtype=np.int64)
    w = np.empty((len(V), K), dtype=np.float64)
    for s in range(0, len(V), 4096):
        blk = V[s:s + 4096]
        dx = blk[:, None, 0] - G[None, :, 0]
        dy = blk[:, None, 1] - G[None, :, 1]
        dz = blk[:, None, 2] - G[None, :, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        order = np.argsort(d2, axis=1, kind="stable")[:, :K + 1]   # ties -> lower index
        d2k = np.take_along_axis(d2, order, axis=1)
        d = np.sqrt(d2k)
        dmax = d[:, K:K + 1]
        with np.errstate(divide="ignore", invalid="ignore"):
            ww = (1.0 - d[:, :K] / dmax) ** 2
        ww = np.where(dmax > 0.0, ww, 0.0)
        sw = ww.sum(axis=1, keepdims=True)
        ww = np.where(sw > 0.0, ww / np.where(sw > 0.0, sw, 1.0), 1.0 / K)
        idx[s:s + 4096] = order[:, :K]
        w[s:s + 4096] = ww
    return idx, w


def node_edges(G32: np.ndarray, k_edges: int = 4) -> np.ndarray:
    """Directed node edges (E,2), sorted by (k, l), symmetric."""
    G = np.asarray(G32, dtype=np.float32).astype(np.float64)
    n = len(G)
    ke = min(k_edges, n - 1)
    adj = set()
    for k in range(n):
        d2 = _sqdist(G, G[k])
        d2[k] = np.inf
        nb = np.argsort(d2, kind="stable")[:ke]
        for l in nb:
            adj.add((k, int(l)))
            adj.add((int(l), k))
    return np.asarray(sorted(adj), dtype=np.int64).reshape(-1, 2)


def edge_weights(material: np.ndarray, node_vid: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """s_kl = mean of the two nodes' material weights (Sec. 3.1)."""
    m = np.asarray(material, dtype=np.float64)[node_vid]
    return 0.5 * (m[edges[:, 0]] + m[edges[:, 1]])


def build_graph(V32: np.ndarray, material: np.ndarray, n_nodes: int, K: int) -> dict:
    """All graph data for one template."""
    vid = farthest_point_sampling(V32, n_nodes)
    G32 = np.asarray(V32, dtype=np.float32)[vid]
    idx, w = bind_vertices(V32, G32, K)
    edges = node_edges(G32)
    s = edge_weights(material, vid, edges)
    return dict(node_vid=vid, bind_idx=idx, bind_w=w, edges=edges, edge_s=s)
