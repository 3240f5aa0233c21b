"""Learned per-node warm start in FP64: features, the MLP, its backward pass
and Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper starts each frame's non-rigid solve from the previous frame's
result (Sec. 3.4, Sec. 4).  The project adds a small network that predicts
each graph node's update so that Gauss-Newton starts closer; plain GN stays
the arbiter (a prediction that raises the energy is rejected).  This module is
the reference the BF16 kernels are checked against.

Network (64 -> 256 -> 256 -> 6, 83,974 parameters), on normalised inputs
x = (f - mu) / sigma:

    h1 = relu(x W1 + b1)        W1: 64 x 256
    h2 = relu(h1 W2 + b2)       W2: 256 x 256
    y  = (h2 W3 + b3) * s_out   W3: 256 x 6      y = (d_omega, d_t)

s_out is a fixed per-output scale (not trained), and mu / sigma / s_out are
fitted to the training rows (``fit_scaling``): column mean and population
standard deviation of the features, root mean square of the targets.

Loss over M rows: L = (1/M) sum_rows ||y - t||^2.  Gradients by the chain
rule; Adam with bias correction (Kingma and Ba, 2015).

The training target of a frame is the update its solve made to each node
(``node_motion``): Log(R_end R_start^T) and t_end - t_start.

Parameter vector order (flat, float): W1 (row-major 64 x 256), b1, W2
(256 x 256), b2, W3 (256 x 6), b3.

Node features (64 per node), pooled at the start point of a frame from the
linearisation there (residuals, per-vertex blocks, flags) over the node's
bound vertices with their binding weights w (W_k = sum of the node's w):

     0- 2  omega_k = Log(R_k)              3- 5  t_k
     6-11  b_k = -(J^T F)_k               12-17  diag(J^T J)_k
    18-23  b_k / (diag_k + tau_k), tau_k = 1e-6 max(diag_k) (+1e-30)
    24-26  sum w r_photo / W_k            27-29  sum w |r_photo| / W_k
    30     sum w r_sil / W_k              31     sum w r_sil^2 / W_k
    32-34  sum w e / W_k                  35-37  sum w |e| / W_k
    38-43  sum w H / W_k (h00 h01 h02 h11 h12 h22)
    44     sum w [visible] / W_k          45     sum w [in B] / W_k
    46     sum w [b = -1] / W_k           47     W_k
    48-50  g_k                            51-56  u_k, the node's update over the previous frame
    57-62  mean of u_l over the node's graph neighbours l (0 without neighbours)
    63     1
(a pooled value is 0 when W_k = 0).
"""
from __future__ import annotations

import numpy as np

D_IN, D_H, D_OUT = 64, 256, 6
N_PARAMS = D_IN * D_H + D_H + D_H * D_H + D_H + D_H * D_OUT + D_OUT   # 83,974


def unpack(theta: np.ndarray):
    """Flat parameter vector -> (W1, b1, W2, b2, W3, b3) views."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    o = 0
    out = []
    for shape in ((D_IN, D_H), (D_H,), (D_H, D_H), (D_H,), (D_H, D_OUT), (D_OUT,)):
        n = int(np.prod(shape))
        out.append(theta[o:o + n].reshape(shape))
        o += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def forward(theta, x, s_out=None):
    """x: M x 64 (normalised features); s_out: 6 output scales (None = 1).
    Returns (y, cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    s = np.ones(D_OUT) if s_out is None else np.asarray(s_out, dtype=np.float64)
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = (h2 @ W3 + b3) * s
    return y, (x, z1, h1, z2, h2, s)


def loss(y, t):
    """L = (1/M) sum ||y - t||^2 and dL/dy."""
    d = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    M = d.shape[0]
    return float((d * d).sum() / max(M, 1)), 2.0 * d / max(M, 1)


def backward(theta, cache, dy):
    """Gradient of L with respect to the flat parameters, given dL/dy."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x, z1, h1, z2, h2, s = cache
    dz3 = np.asarray(dy, dtype=np.float64) * s        # through y = z3 * s_out
    dW3 = h2.T @ dz3
    db3 = dz3.sum(0)
    dh2 = (dz3 @ W3.T) * (z2 > 0.0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2.T) * (z1 > 0.0)
    dW1 = x.T @ dh1
    db1 = dh1.sum(0)
    return pack([dW1, db1, dW2, db2, dW3, db3])


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def fit_scaling(F, T):
    """(mu, sigma, s_out) of training rows F (rows x 64), T (rows x 6):
    column mean and population standard deviation of F (sigma 1 where below
    1e-12; the constant feature 63 keeps mu 0, sigma 1), root mean square of
    each column of T (1 where below 1e-12)."""
    F = np.asarray(F, dtype=np.float64).reshape(-1, D_IN)
    T = np.asarray(T, dtype=np.float64).reshape(-1, D_OUT)
    mu = F.mean(0)
    sigma = F.std(0)
    sigma[sigma < 1e-12] = 1.0
    mu[D_IN - 1], sigma[D_IN - 1] = 0.0, 1.0
    s_out = np.sqrt((T * T).mean(0))
    s_out[s_out < 1e-12] = 1.0
    return mu, sigma, s_out


def node_motion(R_start, t_start, R_end, t_end) -> np.ndarray:
    """Per node (Log(R_end R_start^T), t_end - t_start), n x 6."""
    Rs = np.asarray(R_start, dtype=np.float64).reshape(-1, 3, 3)
    Re = np.asarray(R_end, dtype=np.float64).reshape(-1, 3, 3)
    D = np.einsum("nij,nkj->nik", Re, Rs)
    return np.concatenate([rot_log(D), np.asarray(t_end, dtype=np.float64).reshape(-1, 3)
                           - np.asarray(t_start, dtype=np.float64).reshape(-1, 3)], 1)


# ----------------------------------------------------------------------------
# node features
# ----------------------------------------------------------------------------
def rot_log(R: np.ndarray) -> np.ndarray:
    """Axis-angle of rotation matrices (..., 3, 3), angle in [0, pi)."""
    R = np.asarray(R, dtype=np.float64)
    c = np.clip(0.5 * (np.trace(R, axis1=-2, axis2=-1) - 1.0), -1.0, 1.0)
    th = np.arccos(c)
    v = np.stack([R[..., 2, 1] - R[..., 1, 2], R[..., 0, 2] - R[..., 2, 0], R[..., 1, 0] - R[..., 0, 1]], -1)
    s = np.sin(th)
    f = np.where(th < 1e-7, 0.5, th / (2.0 * np.where(s == 0.0, 1.0, s)))
    return v * f[..., None]


def node_features(R, t, g, rhs, diag, ent_off, ent_vid, ent_w, r_photo, r_sil, e, H, flags,
                  u_prev, edge_off, edge_dst):
    """Features (n x 64) by the definition in the module docstring.

    Per-vertex inputs are those of the linearisation at the start point
    (r_photo N x 3 and r_sil N are zero for inactive vertices; flags carry
    bit 1 visible, 4 in B, 8 b = -1); the node CSR (ent_off, ent_vid, ent_w)
    lists each node's bound vertices with their binding weights."""
    n = len(g)
    F = np.zeros((n, 64))
    F[:, 0:3] = rot_log(np.asarray(R, dtype=np.float64).reshape(n, 3, 3))
    F[:, 3:6] = t
    F[:, 6:12] = rhs
    F[:, 12:18] = diag
    tau = 1e-6 * np.asarray(diag, dtype=np.float64).max(1) + 1e-30
    F[:, 18:24] = rhs / (diag + tau[:, None])
    fl = np.asarray(flags).astype(np.int64)
    per_vertex = np.concatenate([
        r_photo, np.abs(r_photo), np.asarray(r_sil)[:, None], np.asarray(r_sil)[:, None] ** 2,
        e, np.abs(e), H,
        ((fl & 1) != 0)[:, None], ((fl & 4) != 0)[:, None], ((fl & 8) != 0)[:, None]], 1).astype(np.float64)
    for k in range(n):
        a, b = ent_off[k], ent_off[k + 1]
        w = np.asarray(ent_w[a:b], dtype=np.float64)
        W = w.sum()
        F[k, 47] = W
        if W > 0.0:
            F[k, 24:47] = (w[:, None] * per_vertex[ent_vid[a:b]]).sum(0) / W
        nb = edge_dst[edge_off[k]:edge_off[k + 1]]
        if len(nb):
            F[k, 57:63] = np.asarray(u_prev, dtype=np.float64)[nb].mean(0)
    F[:, 48:51] = g
    F[:, 51:57] = u_prev
    F[:, 63] = 1.0
    return F
