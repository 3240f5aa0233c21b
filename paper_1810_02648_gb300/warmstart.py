"""Training and evaluation of the learned warm start (host-side driver).

Every computation runs in the library's kernels (lc_node_features,
lc_solve_nonrigid, lc_mlp_*, lc_warm_start); this module only sequences
them over a capture's frames:

* ``collect``: track a sequence with the plain method (each frame solved from
  the previous frame's result) and record, per frame and node, the features
  at the start and the update the solve converged to: Log(R_end R_start^T)
  and t_end - t_start.
* ``train``: Adam on (features, update) pairs with per-feature
  normalisation, minibatches drawn by a seeded generator.
* ``evaluate``: per frame, the plain solve (n_gn steps) and the warm-started
  solve that stops once it reaches the plain solve's final energy (within a
  relative tolerance), both timed with CUDA events.
"""
from __future__ import annotations

import numpy as np

from .livecap import MLP, MLP_PARAMS


def _rot_log(R):
    R = np.asarray(R, dtype=np.float64)
    c = np.clip(0.5 * (np.trace(R, axis1=-2, axis2=-1) - 1.0), -1.0, 1.0)
    th = np.arccos(c)
    v = np.stack([R[..., 2, 1] - R[..., 1, 2], R[..., 0, 2] - R[..., 2, 0], R[..., 1, 0] - R[..., 0, 1]], -1)
    s = np.sin(th)
    f = np.where(th < 1e-7, 0.5, th / (2.0 * np.where(s == 0.0, 1.0, s)))
    return v * f[..., None]


def node_update(start: dict, end: dict) -> np.ndarray:
    """(Log(R_end R_start^T), t_end - t_start) per node, n x 6."""
    Rd = np.einsum("nij,nkj->nik", end["R"].astype(np.float64), start["R"].astype(np.float64))
    return np.concatenate([_rot_log(Rd), end["t"].astype(np.float64) - start["t"]], 1)


def _upload(ctx, frame):
    rgb, dt, mask = frame
    ctx.upload_frame(rgb, dt, np.asarray(mask, dtype=np.uint8), None, None)


def collect(ctx, frames):
    """Plain tracking of ``frames`` (list of (rgb, dt, mask)) from the
    context's current node parameters.  Returns features (T, n, 64),
    targets (T, n, 6) and the plain final energies (T)."""
    F, Tg, E = [], [], []
    for fr in frames:
        _upload(ctx, fr)
        start = ctx.read_back(V=False, flags=False)
        ctx.compute_visibility()
        F.append(ctx.node_features())
        st = ctx.solve_nonrigid()
        end = ctx.read_back(V=False, flags=False)
        Tg.append(node_update(start, end))
        E.append(st["e_total"])
        ctx.record_motion()
    return np.stack(F), np.stack(Tg).astype(np.float32), np.array(E)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (flat layout of LC_MLP_PARAMS)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / 64), size=64 * 256), np.zeros(256),
             rng.normal(0.0, np.sqrt(2.0 / 256), size=256 * 256), np.zeros(256),
             rng.normal(0.0, np.sqrt(1.0 / 256), size=256 * 6), np.zeros(6)]
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == MLP_PARAMS
    return theta


def train(F, T, steps: int, batch: int = 1024, lr: float = 1e-3, seed: int = 0, device: int = 0,
          target_scale: float | None = None, log_every: int = 0):
    """Adam on rows of F (rows x 64) / T (rows x 6).  Targets are scaled by
    1 / target_scale inside the loss (the network's output is scaled back by
    the caller through ``Predictor``).  Returns (Predictor, losses)."""
    import torch
    F = np.asarray(F, dtype=np.float32).reshape(-1, 64)
    T = np.asarray(T, dtype=np.float32).reshape(-1, 6)
    mu = F.mean(0)
    sigma = F.std(0)
    sigma[sigma < 1e-12] = 1.0
    mu[63], sigma[63] = 0.0, 1.0                      # keep the constant feature as is
    s = float(target_scale) if target_scale else float(np.abs(T).std() + 1e-12)
    net = MLP(device, init_params(seed), mu, sigma)
    Fd = torch.from_numpy(F).to(f"cuda:{device}")
    Td = torch.from_numpy(T / s).to(f"cuda:{device}")
    rng = np.random.default_rng(seed + 1)
    losses = []
    rows = F.shape[0]
    for k in range(steps):
        idx = rng.integers(0, rows, size=min(batch, rows)).astype(np.int32)
        want = log_every and (k % log_every == 0 or k == steps - 1)
        L = net.train_step(Fd, Td, idx, lr, want_loss=bool(want))
        if want:
            losses.append((k, L))
    return Predictor(net, s), losses


class Predictor:
    """The trained network plus the scale of its targets: the output layer is
    rescaled in place so that the network predicts the update directly."""

    def __init__(self, net: MLP, scale: float):
        theta = net.params()
        theta[-6 - 256 * 6:] *= scale                  # W3 and b3
        self.net = MLP(net.device, theta, *self._norm(net))
        self.scale = scale
        net.close()

    @staticmethod
    def _norm(net):
        return net._keep[1], net._keep[2]

    def close(self):
        self.net.close()


def evaluate(plain_ctx, warm_ctx, pred: Predictor, frames, streams, rel_tol: float = 1e-4):
    """Plain vs warm-started solves along the plain trajectory.

    ``plain_ctx`` runs its n_gn steps from the previous frame's result;
    ``warm_ctx`` (same capture, normally a larger n_gn budget) starts from
    the same parameters, applies the network's prediction (kept only if it
    does not raise the energy) and runs Gauss-Newton until its energy is
    within rel_tol of the plain solve's final energy (the solve's
    target-energy stop).  Both are timed with CUDA events on their streams
    (``streams`` = (plain, warm) torch streams).  Returns per-frame records."""
    import torch
    out = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    sp, sw = streams
    for fr in frames:
        _upload(plain_ctx, fr)
        _upload(warm_ctx, fr)
        start = plain_ctx.read_back(V=False, flags=False)
        n = start["R"].shape[0]
        torch.cuda.synchronize()
        ev[0].record(sp)
        plain_ctx.solve_nonrigid(stats=False)
        ev[1].record(sp)
        torch.cuda.synchronize()
        plain_stats = plain_ctx.read_stats()
        plain = plain_ctx.read_back(V=False, flags=False)
        e_plain = plain_stats["e_total"]
        warm_ctx.set_node_params(start["R"].reshape(n, 9), start["t"])
        warm_ctx.set_params(target_energy=float(e_plain) * (1.0 + rel_tol))
        torch.cuda.synchronize()
        ev[2].record(sw)
        warm_ctx.warm_start(pred.net, sync=False)
        warm_ctx.solve_nonrigid(stats=False)
        ev[3].record(sw)
        torch.cuda.synchronize()
        st = warm_ctx.read_stats()
        out.append(dict(plain_ms=ev[0].elapsed_time(ev[1]), warm_ms=ev[2].elapsed_time(ev[3]),
                        e_plain=e_plain, e_warm=st["e_total"], steps_plain=plain_stats["n_gn_done"],
                        steps_warm=st["n_gn_done"],
                        reached=bool(st["e_total"] <= e_plain * (1.0 + rel_tol))))
        # both continue along the plain trajectory
        warm_ctx.set_node_params(plain["R"].reshape(n, 9), plain["t"])
        plain_ctx.record_motion()
        warm_ctx.record_motion()
    return out
