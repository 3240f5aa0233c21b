"""Training and evaluation of the learned warm start (host-side driver).

Every computation runs in the library's kernels (lc_node_features,
lc_solve_nonrigid, lc_record_motion / lc_read_motion, lc_mlp_*,
lc_warm_start); this module only sequences them over a capture's frames and
keeps the results in device memory:

* ``collect``: track a sequence with the plain method (each frame solved from
  the previous frame's result) and record, per frame and node, the features
  at the start and the update the solve made (the motion recorded after it:
  Log(R_end R_start^T), t_end - t_start).
* ``train``: the network's input normalisation and output scale fitted to the
  rows on the device, then Adam on minibatches drawn by a seeded generator.
* ``evaluate``: per frame, the plain method's energy after its full step
  budget is the target; the plain solve from the previous frame's result and
  the warm-started solve then both run with the same target-energy stop, and
  both are timed with CUDA events.
"""
from __future__ import annotations

import numpy as np

from .livecap import MLP, MLP_PARAMS


def _upload(ctx, frame):
    """frame: (rgb, dt, mask) or (rgb, dt, mask, joints2d, joints3d)."""
    rgb, dt, mask = frame[:3]
    j2, j3 = (frame[3], frame[4]) if len(frame) > 3 else (None, None)
    ctx.upload_frame(rgb, dt, np.asarray(mask, dtype=np.uint8), j2, j3)


def restart(ctx, pose: bool = False):
    """Start a new sequence: identity node parameters and zero motion; with
    ``pose``, the pose stage restarts from the pose last set and forgets its
    recorded frames."""
    ctx.set_node_params(None, None)
    ctx.record_motion()
    ctx.record_motion()
    if pose:
        ctx.reset_pose()
        ctx.pose_clear_history()


def collect(ctx, frames, skip: int = 0, pose: bool = False, euler: bool = True, from_identity: bool = False):
    """Plain tracking of ``frames`` (an iterable of (rgb, dt, mask), with
    joints when ``pose``) from the context's current state.  With ``pose``
    every frame first runs the pose stage (from the explicit Euler start once
    a frame is recorded, with ``euler``, else from the last solved pose) and
    ends with lc_pose_advance.  With ``from_identity`` the non-rigid stage of
    every frame starts from the identity (the motion is recorded there, so
    the target is the update from that start).
    Returns features (T, n, 64) and targets (T, n, 6) as device tensors and
    the plain final energies (T) of the frames after the first ``skip``
    (those are tracked but not kept)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    F, Tg, E = [], [], []
    for i, fr in enumerate(frames):
        _upload(ctx, fr)
        if pose:
            if euler and i > 0:
                ctx.pose_extrapolate()
            ctx.solve_pose(stats=False)
        if from_identity:
            ctx.set_node_params(None, None)
            ctx.record_motion()
        keep = i >= skip
        if keep:
            ctx.compute_visibility()
            f = torch.empty((ctx.n, 64), dtype=torch.float32, device=dev)
            ctx.node_features(out=f)
        st = ctx.solve_nonrigid()
        ctx.record_motion()
        if pose:
            ctx.pose_advance()
        if keep:
            u = torch.empty((ctx.n, 6), dtype=torch.float32, device=dev)
            ctx.read_motion(out=u)
            F.append(f)
            Tg.append(u)
            E.append(st["e_total"])
    if not F:
        return (torch.empty((0, ctx.n, 64), device=dev), torch.empty((0, ctx.n, 6), device=dev), np.zeros(0))
    return torch.stack(F), torch.stack(Tg), np.array(E)


def keep_converged(F, T, E, factor: float = 100.0):
    """The training frames whose plain solve converged: final energy finite
    and at most ``factor`` times the median final energy of the set, targets
    finite.  A tracked solve that ran away from the capture (Gauss-Newton
    without step control can, on a rare frame) would otherwise put its
    motion, orders of magnitude off, among the targets.  Returns (F, T,
    kept mask over the frames)."""
    import torch
    E = np.asarray(E, dtype=np.float64)
    ok = np.isfinite(E)
    if ok.any():
        ok &= E <= factor * np.median(E[ok])
    fin = torch.isfinite(T.reshape(T.shape[0], -1)).all(1).cpu().numpy()
    keep = ok & fin
    idx = torch.as_tensor(np.nonzero(keep)[0], device=F.device)
    return F.index_select(0, idx), T.index_select(0, idx), keep


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
          log_every: int = 0):
    """Adam on the rows of F (device, rows x 64) / T (device, rows x 6) after
    fitting the network's scaling to them (lc_mlp_fit_scaling).  Returns
    (network, losses)."""
    F = F.reshape(-1, 64).contiguous()
    T = T.reshape(-1, 6).contiguous()
    net = MLP(device, init_params(seed))
    net.fit_scaling(F, T)
    rng = np.random.default_rng(seed + 1)
    losses = []
    rows = F.shape[0]
    for k in range(steps):
        idx = rng.integers(0, rows, size=min(batch, rows)).astype(np.int32)
        want = log_every and (k % log_every == 0 or k == steps - 1)
        L = net.train_step(F, T, idx, lr, want_loss=bool(want))
        if want:
            losses.append((k, L))
    return net, losses


def evaluate(plain_ctx, warm_ctx, net: MLP, frames, streams, rel_tol: float = 1e-4):
    """Plain vs warm-started solves along the plain trajectory, with one
    stopping rule for both.

    Per frame: an untimed reference solve of ``plain_ctx`` (its full n_gn
    steps from the previous frame's result: a target below every energy)
    gives the energy E* that the plain method reaches.  Then, from the same
    start and with the target-energy stop at E* (1 + rel_tol): the plain
    solve (``plain_ctx``) and the warm-started one (``warm_ctx``, normally a
    larger step budget: the network's prediction, kept only if it does not
    raise the energy, then Gauss-Newton), each timed with CUDA events on its
    stream (``streams`` = (plain, warm) torch streams).  Every solve runs
    with a target, so the captured graphs are reused (only the target's
    value changes); the warm arm runs once untimed on the first frame to
    capture its graphs.  Both contexts continue from the reference solve's
    result.  Returns per-frame records."""
    import torch
    out = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    sp, sw = streams
    never = 1e-30
    for k, fr in enumerate(frames):
        _upload(plain_ctx, fr)
        _upload(warm_ctx, fr)
        start = plain_ctx.read_back(V=False, flags=False)
        n = start["R"].shape[0]
        if k == 0:
            warm_ctx.set_params(target_energy=never)
            warm_ctx.set_node_params(start["R"].reshape(n, 9), start["t"])
            warm_ctx.warm_start(net, sync=False)
            warm_ctx.solve_nonrigid(stats=False)
        plain_ctx.set_params(target_energy=never)
        ref = plain_ctx.solve_nonrigid()
        end = plain_ctx.read_back(V=False, flags=False)
        e_star = float(ref["e_total"])
        target = e_star * (1.0 + rel_tol)
        # plain, same start, target stop
        plain_ctx.set_node_params(start["R"].reshape(n, 9), start["t"])
        plain_ctx.set_params(target_energy=target)
        torch.cuda.synchronize()
        ev[0].record(sp)
        plain_ctx.solve_nonrigid(stats=False)
        ev[1].record(sp)
        torch.cuda.synchronize()
        ps = plain_ctx.read_stats()
        # warm start + Gauss-Newton, same start, same target stop
        warm_ctx.set_node_params(start["R"].reshape(n, 9), start["t"])
        warm_ctx.set_params(target_energy=target)
        torch.cuda.synchronize()
        ev[2].record(sw)
        warm_ctx.warm_start(net, sync=False)
        warm_ctx.solve_nonrigid(stats=False)
        ev[3].record(sw)
        torch.cuda.synchronize()
        ws = warm_ctx.read_stats()
        e0_plain, e0_warm = ps["e_gn_all"][0], ws["e_gn_all"][0]
        out.append(dict(plain_ms=ev[0].elapsed_time(ev[1]), warm_ms=ev[2].elapsed_time(ev[3]),
                        e_star=e_star, e_plain=ps["e_total"], e_warm=ws["e_total"],
                        steps_ref=ref["n_gn_done"], steps_plain=ps["n_gn_done"], steps_warm=ws["n_gn_done"],
                        e_start=e0_plain, e_predicted=e0_warm, kept=bool(e0_warm < e0_plain),
                        reached_plain=bool(ps["e_total"] <= target), reached_warm=bool(ws["e_total"] <= target)))
        # both continue along the plain trajectory
        for c in (plain_ctx, warm_ctx):
            c.set_node_params(end["R"].reshape(n, 9), end["t"])
            c.record_motion()
    return out


def summary(res) -> dict:
    """Frames/s of both arms over the records of ``evaluate`` and the
    step counts (the warm arm's unreached frames count with their time)."""
    plain_ms = float(np.sum([r["plain_ms"] for r in res]))
    warm_ms = float(np.sum([r["warm_ms"] for r in res]))
    return dict(frames=len(res), plain_frames_per_s=len(res) / (plain_ms / 1e3),
                warm_frames_per_s=len(res) / (warm_ms / 1e3), gain=plain_ms / warm_ms,
                reached_plain=float(np.mean([r["reached_plain"] for r in res])),
                reached_warm=float(np.mean([r["reached_warm"] for r in res])),
                kept=float(np.mean([r["kept"] for r in res])),
                steps_plain_mean=float(np.mean([r["steps_plain"] for r in res])),
                steps_warm_mean=float(np.mean([r["steps_warm"] for r in res])),
                steps_warm_median=float(np.median([r["steps_warm"] for r in res])),
                start_energy_ratio_median=float(np.median([r["e_predicted"] / r["e_start"] for r in res])))
