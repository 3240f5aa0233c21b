"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import json
import os

import numpy as np

from oracle import nonrigid as onr
from oracle import visibility as ovis

REPORT = {}


def report(key, **vals):
    """Record observed error figures; written to $LC_REPORT_DIR if set."""
    REPORT[key] = {k: float(v) if np.isscalar(v) else v for k, v in vals.items()}
    d = os.environ.get("LC_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "parity_report.json"), "w") as f:
            json.dump(REPORT, f, indent=1, sort_keys=True)


def csr_edges(g):
    off, dst = g["edge_off"], g["edge_dst"]
    src = np.repeat(np.arange(len(off) - 1), np.diff(off))
    return np.stack([src, dst], 1).astype(np.int64)


def graph_from_gpu(g):
    return dict(node_vid=g["node_vid"].astype(np.int64), bind_idx=g["bind_idx"].astype(np.int64),
                bind_w=g["bind_w"], edges=csr_edges(g), edge_s=g["edge_s"])


def oracle_problem(scene, g, flags=None, base32=None):
    P = onr.problem_from_scene(scene, graph_from_gpu(g), base32)
    if flags is not None:
        set_flags(P, flags)
    return P


def set_flags(P, flags):
    P.vis = (flags & ovis.FLAG_VISIBLE) != 0
    P.inB = (flags & ovis.FLAG_INB) != 0
    P.bsign = np.where((flags & ovis.FLAG_BNEG) != 0, -1.0, 1.0)


def random_params(n, seed, rot=0.05, trans=0.005):
    rng = np.random.default_rng(seed)
    R = onr.so3_exp(rng.normal(scale=rot, size=(n, 3))).astype(np.float32)
    t = rng.normal(scale=trans, size=(n, 3)).astype(np.float32)
    return R, t


def vec6(x):
    return np.asarray(x, dtype=np.float64).reshape(-1)


def oracle_vertex_blocks(P, v32, uv32):
    """Residuals and A_i^T A_i, A_i^T r_i at given FP32 warped positions and
    projections (the inputs of the GPU's residual kernel), in FP64."""
    v = v32.astype(np.float64)
    u, w = uv32[:, 0].astype(np.float64), uv32[:, 1].astype(np.float64)
    ok = (v[:, 2] > 1e-3) & (u >= 0) & (u <= P.W - 1) & (w >= 0) & (w <= P.H - 1)
    ph = ok & P.vis
    si = ok & P.inB
    (gxI, gyI), (gxD, gyD) = P.grads()
    Dp = onr.dproj(P, v)
    N = len(v)
    r_photo = np.zeros((N, 3))
    r_sil = np.zeros(N)
    H = np.zeros((N, 3, 3))
    e = np.zeros((N, 3))
    ip = np.nonzero(ph)[0]
    if len(ip):
        r_photo[ip] = np.sqrt(P.w_photo) * (onr.bilinear(P.rgb, u[ip], w[ip]) - P.albedo[ip])
        G = np.stack([onr.bilinear(gxI, u[ip], w[ip]), onr.bilinear(gyI, u[ip], w[ip])], 2)
        A = np.sqrt(P.w_photo) * (G @ Dp[ip])
        H[ip] += np.einsum("nri,nrj->nij", A, A)
        e[ip] += np.einsum("nri,nr->ni", A, r_photo[ip])
    isl = np.nonzero(si)[0]
    if len(isl):
        r_sil[isl] = np.sqrt(P.w_sil) * onr.bilinear(P.dt, u[isl], w[isl])
        G = np.stack([onr.bilinear(gxD, u[isl], w[isl]), onr.bilinear(gyD, u[isl], w[isl])], 1)[:, None, :]
        A = (np.sqrt(P.w_sil) * P.bsign[isl])[:, None, None] * (G @ Dp[isl])
        H[isl] += np.einsum("nri,nrj->nij", A, A)
        e[isl] += A[:, 0, :] * r_sil[isl, None]
    H6 = np.stack([H[:, 0, 0], H[:, 0, 1], H[:, 0, 2], H[:, 1, 1], H[:, 1, 2], H[:, 2, 2]], 1)
    return dict(r_photo=r_photo, r_sil=r_sil, H=H6, e=e, photo_on=ph, sil_on=si)
