"""GPU parity of the learned warm start: the BF16 network (forward, gradient,
Adam) against the FP64 oracle, the node features against the oracle's
pooling at identical inputs, the accept / reject rule, and the solve's stop
at a target energy.

BF16 tolerances.  The kernels round the normalised inputs, the weights, the
hidden activations and the back-propagated gradients to BF16 (8 significant
bits, unit roundoff 2^-9) and accumulate in FP32.  The test emulates exactly
those roundings in FP64 (``_emulate``): the kernels must match the emulation
to FP32 accumulation error (a rounding that flips at a BF16 tie moves one
element by one BF16 ulp), and the emulation must stay within the BF16 bound
of the unrounded FP64 network (two rounded activation layers: a few 2^-9
relative on the output's scale).
"""
import numpy as np
import pytest

import synth
from gpu_helpers import random_params, report
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _net(seed, M, scale=0.15):
    rng = np.random.default_rng(seed)
    theta = rng.normal(scale=scale, size=omlp.N_PARAMS).astype(np.float32)
    mu = rng.normal(size=64).astype(np.float32)
    sigma = rng.uniform(0.5, 2.0, size=64).astype(np.float32)
    F = (rng.normal(size=(M, 64)) * sigma + mu).astype(np.float32)
    T = rng.normal(scale=0.3, size=(M, 6)).astype(np.float32)
    return theta, mu, sigma, F, T


def _emulate(theta, mu, sigma, F, T, s_out=None):
    """The kernels' precision choices in FP64: returns (y, loss, grad)."""
    W1, b1, W2, b2, W3, b3 = omlp.unpack(theta.astype(np.float64))
    W1, W2, W3 = bf16(W1), bf16(W2), bf16(W3)
    so = np.ones(6) if s_out is None else np.asarray(s_out, dtype=np.float64)
    M = F.shape[0]
    X = bf16((F.astype(np.float32) - mu) / sigma)
    H1 = bf16(np.maximum(X @ W1 + b1, 0.0))
    H2 = bf16(np.maximum(H1 @ W2 + b2, 0.0))
    y = (H2 @ W3 + b3) * so
    d = y - T
    dY = 2.0 * d / M * so
    dYb = bf16(dY)
    gW3 = H2.T @ dYb
    gb3 = dY.sum(0)
    dZ2 = bf16((dYb @ W3.T) * (H2 > 0))
    gW2 = H1.T @ dZ2
    gb2 = dZ2.sum(0)
    dZ1 = bf16((dZ2 @ W2.T) * (H1 > 0))
    gW1 = X.T @ dZ1
    gb1 = dZ1.sum(0)
    return y, float((d * d).sum() / M), omlp.pack([gW1, gb1, gW2, gb2, gW3, gb3])


def _blocks(v):
    return omlp.unpack(np.asarray(v, dtype=np.float64))


S_OUT = np.array([0.02, 0.5, 1.0, 3e-3, 2.0, 7e-4], np.float32)


@pytest.mark.parametrize("gemm", [0, 1], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("M,scaled", [(1, False), (37, False), (500, False), (2053, False), (500, True)])
def test_forward_matches_oracle(M, scaled, gemm):
    from paper_1810_02648_gb300 import MLP
    theta, mu, sigma, F, T = _net(1, M)
    net = MLP(0, theta, mu, sigma)
    net.set_gemm(gemm)
    s_out = S_OUT if scaled else None
    if scaled:
        net.set_scaling(s_out=s_out)
    y = net.forward(F)
    y_em, _, _ = _emulate(theta, mu, sigma, F, T, s_out)
    x = (F.astype(np.float64) - mu) / sigma
    y64, _ = omlp.forward(theta.astype(np.float64), x, s_out)
    # per output column: the scales differ by orders of magnitude
    scale = np.abs(y64).max(0)
    d_em = (np.abs(y - y_em) / scale).max()
    d_64 = (np.abs(y_em - y64) / scale).max()
    report(f"mlp_forward_{M}{'_scaled' if scaled else ''}_g{gemm}", vs_emulation=d_em, emulation_vs_fp64=d_64)
    assert d_em <= 2e-3       # FP32 accumulation; rare BF16 tie flips
    assert d_64 <= 4e-2       # two BF16 activation layers + BF16 weights
    net.close()


@pytest.mark.parametrize("gemm", [0, 1], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("M,scaled", [(64, False), (1000, False), (1000, True), (4096, False)])
def test_gradient_matches_oracle(M, scaled, gemm):
    from paper_1810_02648_gb300 import MLP
    theta, mu, sigma, F, T = _net(2, M)
    s_out = S_OUT if scaled else None
    if scaled:
        T = (T * S_OUT).astype(np.float32)           # targets on the outputs' scales
    net = MLP(0, theta, mu, sigma)
    net.set_gemm(gemm)
    if scaled:
        net.set_scaling(s_out=s_out)
    g, L = net.gradient(F, T)
    _, L_em, g_em = _emulate(theta, mu, sigma, F, T, s_out)
    x = (F.astype(np.float64) - mu) / sigma
    y64, cache = omlp.forward(theta.astype(np.float64), x, s_out)
    L64, dy = omlp.loss(y64, T)
    g64 = omlp.backward(theta.astype(np.float64), cache, dy)
    errs = {}
    for name, a, b, c in zip(["W1", "b1", "W2", "b2", "W3", "b3"], _blocks(g), _blocks(g_em), _blocks(g64)):
        errs[name] = (np.linalg.norm(a - b) / np.linalg.norm(b), np.linalg.norm(b - c) / np.linalg.norm(c))
    report(f"mlp_gradient_{M}{'_scaled' if scaled else ''}_g{gemm}", loss_rel=abs(L - L_em) / L_em,
           **{f"{k}_vs_em": v[0] for k, v in errs.items()}, **{f"{k}_em_vs_fp64": v[1] for k, v in errs.items()})
    assert abs(L - L_em) <= 1e-4 * L_em and abs(L_em - L64) <= 5e-2 * L64
    for name, (e_em, e_64) in errs.items():
        assert e_em <= 5e-3, name
        assert e_64 <= 8e-2, name
    net.close()


def test_adam_step_matches_oracle():
    """First Adam step: every parameter moves by lr times the sign of its
    gradient (bias-corrected moments), so the update is pinned by the
    gradient's signs."""
    import torch
    from paper_1810_02648_gb300 import MLP
    theta, mu, sigma, F, T = _net(3, 256)
    net = MLP(0, theta, mu, sigma)
    g, _ = net.gradient(F, T)
    Fd = torch.from_numpy(F).cuda()
    Td = torch.from_numpy(T).cuda()
    idx = np.arange(256, dtype=np.int32)
    lr = 1e-3
    L = net.train_step(Fd, Td, idx, lr, want_loss=True)
    step = net.params().astype(np.float64) - theta
    nz = np.abs(g) > 1e-3                        # eps = 1e-8 is negligible against |g| here
    expect = -lr * np.sign(g)
    report("mlp_adam", loss=L, max_dev=np.abs(step[nz] - expect[nz]).max())
    assert np.allclose(step[nz], expect[nz], rtol=0, atol=2e-6)
    # a few more steps on the same batch reduce the loss
    for _ in range(20):
        net.train_step(Fd, Td, idx, lr)
    L2 = net.train_step(Fd, Td, idx, lr, want_loss=True)
    assert L2 < L
    net.close()


@pytest.mark.parametrize("rows", [1, 777, 300001])
def test_fit_scaling_matches_oracle(rows):
    """Column moments on the device (FP64, fixed order) against the oracle's
    definition on the same rows; the set / get round trip."""
    import torch
    from paper_1810_02648_gb300 import MLP
    rng = np.random.default_rng(rows)
    F = (rng.normal(size=(rows, 64)) * rng.uniform(1e-3, 30.0, size=64) + rng.normal(scale=5.0, size=64))
    F[:, 63] = 1.0
    F[:, 7] = -2.5
    F = F.astype(np.float32)
    T = (rng.normal(size=(rows, 6)) * np.array([0.02, 0.03, 0.01, 2e-3, 1e-3, 5e-3])).astype(np.float32)
    T[:, 4] = 0.0
    net = MLP(0)
    net.fit_scaling(torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda())
    mu, sigma, s_out = net.scaling()
    rmu, rsig, rs = omlp.fit_scaling(F, T)
    d_mu = (np.abs(mu - rmu) / rsig).max()
    d_sig = (np.abs(sigma - rsig) / rsig).max()
    d_s = (np.abs(s_out - rs) / rs).max()
    report(f"mlp_fit_scaling_{rows}", mu=d_mu, sigma=d_sig, s_out=d_s)
    # FP64 moments rounded once to FP32 (a mean of ~15 against a deviation
    # of ~0.1 moves by up to half an FP32 ulp of the mean); a single row has
    # sigma 1 everywhere
    ulp = np.spacing(np.abs(rmu).astype(np.float32)).astype(np.float64)
    assert (np.abs(mu - rmu) <= ulp + 1e-7 * rsig).all()
    assert d_sig <= 1e-6 and d_s <= 1e-6
    assert mu[63] == 0.0 and sigma[63] == 1.0 and s_out[4] == 1.0 and sigma[7] == 1.0
    net.set_scaling(mu=rmu.astype(np.float32) + 1, sigma=None, s_out=np.full(6, 3.0, np.float32))
    mu2, sigma2, s2 = net.scaling()
    assert np.array_equal(mu2, rmu.astype(np.float32) + 1) and np.array_equal(sigma2, sigma)
    assert np.all(s2 == 3.0)
    net.close()


def _ctx(scene, **params):
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    ctx = Context(0)
    setup_scene(ctx, scene)
    if params:
        ctx.set_params(**params)
    return ctx


def test_node_features_match_oracle():
    tiny = synth.make_scene("tiny")
    ctx = _ctx(tiny)
    n = tiny.n_nodes
    RA, tA = random_params(n, 21)
    ctx.set_node_params(RA.reshape(n, 9), tA)
    ctx.record_motion()                         # motion from the identity to A
    RB, tB = random_params(n, 22)
    ctx.set_node_params(RB.reshape(n, 9), tB)
    ctx.compute_visibility()
    F = ctx.node_features()
    lin = ctx.eval_linearization()
    rhs, diag = ctx.eval_gradient()
    flags = ctx.read_visibility()["flags"]
    g = ctx.read_graph()
    N, K = tiny.N, tiny.K
    order = np.lexsort((np.repeat(np.arange(N), K), g["bind_idx"].ravel()))
    ent_node = g["bind_idx"].ravel()[order]
    ent_vid = np.repeat(np.arange(N), K)[order]
    ent_w = g["bind_w"].ravel()[order]
    ent_off = np.searchsorted(ent_node, np.arange(n + 1))
    u_prev = np.concatenate([omlp.rot_log(RA.astype(np.float64)), tA], 1)
    gpos = tiny.V[g["node_vid"]]
    ref = omlp.node_features(RB.reshape(n, 9), tB, gpos, rhs.reshape(n, 6), diag.reshape(n, 6), ent_off, ent_vid,
                             ent_w, lin["r_photo"], lin["r_sil"], lin["e"], lin["H"], flags, u_prev,
                             g["edge_off"], g["edge_dst"])
    scale = np.maximum(np.abs(ref).max(0), 1e-6)
    d = (np.abs(F - ref) / scale).max(0)
    report("node_features", max_rel=d.max(), worst_feature=int(d.argmax()))
    assert d.max() <= 1e-4
    ctx.close()


def test_read_motion_matches_oracle():
    """The recorded motion between two parameter sets (the training target)
    against the oracle's Log(R_end R_start^T), t_end - t_start."""
    tiny = synth.make_scene("tiny")
    ctx = _ctx(tiny)
    n = tiny.n_nodes
    RA, tA = random_params(n, 41)
    ctx.set_node_params(RA.reshape(n, 9), tA)
    ctx.record_motion()
    a = ctx.read_back(V=False, flags=False)
    RB, tB = random_params(n, 42)
    ctx.set_node_params(RB.reshape(n, 9), tB)
    ctx.record_motion()
    b = ctx.read_back(V=False, flags=False)
    u = ctx.read_motion()
    ref = omlp.node_motion(a["R"], a["t"], b["R"], b["t"])
    d = np.abs(u - ref).max()
    report("read_motion", max_abs=d, max_ref=np.abs(ref).max())
    # FP32 products and arccos near small angles: 1e-5 rad absolute
    assert d <= 1e-5
    ctx.close()


def test_warm_start_accepts_and_rejects():
    """A network that predicts zero leaves the parameters and the energy
    unchanged (accepted: not higher); one that predicts a large rotation
    raises the energy and is rejected, restoring the start exactly."""
    from paper_1810_02648_gb300 import MLP
    tiny = synth.make_scene("tiny")
    ctx = _ctx(tiny)
    n = tiny.n_nodes
    R, t = random_params(n, 31)
    ctx.set_node_params(R.reshape(n, 9), t)
    start = ctx.read_back(V=False, flags=False)
    zero = MLP(0)
    acc, e = ctx.warm_start(zero)
    after = ctx.read_back(V=False, flags=False)
    assert acc and e[1] == e[0]
    assert np.array_equal(after["R"], start["R"]) and np.array_equal(after["t"], start["t"])
    theta = np.zeros(omlp.N_PARAMS, np.float32)
    theta[-6:] = [1.0, 0.5, 0.0, 0.05, 0.0, 0.0]           # b3: a large update for every node
    bad = MLP(0, theta)
    acc2, e2 = ctx.warm_start(bad)
    after2 = ctx.read_back(V=False, flags=False)
    report("warm_start_rules", e_start=e2[0], e_bad=e2[1])
    assert not acc2 and e2[1] > e2[0]
    assert np.array_equal(after2["R"], start["R"]) and np.array_equal(after2["t"], start["t"])
    zero.close()
    bad.close()
    ctx.close()


def test_solve_stops_at_target_energy():
    tiny = synth.make_scene("tiny")
    ctx = _ctx(tiny, n_pcg=3)
    full = ctx.solve_nonrigid()
    hist = np.array(full["e_gn_all"][:tiny.n_gn])
    target = float(hist[2]) * (1 + 1e-6)          # reached at the third linearisation at the latest
    stop = int(np.nonzero(hist <= target)[0][0])
    ctx.set_params(n_pcg=3, target_energy=target, gn_block=1)
    ctx.set_node_params(None, None)
    st = ctx.solve_nonrigid()
    report("target_energy", n_gn_done=st["n_gn_done"], e_total=st["e_total"], target=target, stop=stop)
    assert st["n_gn_done"] == stop
    assert abs(st["e_total"] - hist[stop]) <= 1e-9 * hist[stop]
    assert st["e_gn_all"][:stop + 1] == full["e_gn_all"][:stop + 1]
    # with gn_block 1 the steps after the first are conditional graph nodes:
    # the stopped solve launched only the steps it took
    assert full["n_kernels_step"] == 0 and st["n_kernels_step"] > 0
    # a target below every energy: the chain of conditional steps runs them
    # all, bit-identical to the unrolled solve
    ctx.set_params(n_pcg=3, target_energy=float(hist.min()) * 0.5, gn_block=2)
    ctx.set_node_params(None, None)
    never = ctx.solve_nonrigid()
    out_never = ctx.read_back(flags=False)
    assert never["n_gn_done"] == tiny.n_gn and never["e_gn_all"] == full["e_gn_all"]
    assert never["e_total"] == full["e_total"]
    # switching the target off restores the unrolled solve
    ctx.set_params(n_pcg=3, target_energy=0.0)
    ctx.set_node_params(None, None)
    assert ctx.solve_nonrigid()["e_total"] == full["e_total"]
    out_full = ctx.read_back(flags=False)
    assert np.array_equal(out_full["R"], out_never["R"]) and np.array_equal(out_full["V"], out_never["V"])
    ctx.close()


def _render_seq(args):
    import synth as _synth
    s, n_frames = args
    scene = _synth.make_scene("tiny")
    Vs = _synth.ar1_sequence(scene.V, n_frames, 64, 0.05, 0.01, seed=s)
    return [_synth.render_frame(v, scene.F, scene.albedo, scene.cam, seed=10000 * s + i) for i, v in enumerate(Vs)]


def _tiny_sequences(seeds, n_frames):
    import multiprocessing as mp
    import os
    with mp.get_context("spawn").Pool(min(len(seeds), os.cpu_count() or 1)) as pool:
        return pool.map(_render_seq, [(s, n_frames) for s in seeds])


def _restart(ctx):
    ctx.set_node_params(None, None)
    ctx.record_motion()
    ctx.record_motion()          # motion zero: the previous state is the identity too


def test_learned_warm_start_gain():
    """Train on tracked AR(1) sequences of the capsule (control-point motion
    rho 0.9), evaluate on a held-out sequence with one stopping rule for
    both arms: per frame the plain method's own energy after its full step
    budget is the target, and the plain solve from the previous frame's
    result and the warm-started solve (up to twice the budget) both stop
    there.  The plain arm reaches its own target on every frame by
    construction (a check of the protocol); the warm arm's reach, step
    counts and frames/s ratio are recorded."""
    import torch
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    from paper_1810_02648_gb300 import warmstart as ws
    tiny = synth.make_scene("tiny")
    seqs = _tiny_sequences(list(range(1, 41)) + [999], 41)
    train_seqs, eval_seq = seqs[:-1], seqs[-1]
    sp, sw = torch.cuda.Stream(), torch.cuda.Stream()
    plain = Context(0, stream=sp)
    setup_scene(plain, tiny)
    plain.set_params(gn_block=1)
    Fs, Ts = [], []
    for seq in train_seqs:
        _restart(plain)
        F, T, _ = ws.collect(plain, seq, skip=1)   # the first frame starts from the identity
        Fs.append(F)
        Ts.append(T)
    net, losses = ws.train(torch.cat(Fs), torch.cat(Ts), steps=4000, batch=2048, lr=1e-3, seed=0, log_every=500)
    warm = Context(0, stream=sw)
    setup_scene(warm, tiny)
    warm.set_params(n_gn=2 * tiny.n_gn, gn_block=1)
    for c in (plain, warm):
        _restart(c)
    ws.collect(plain, eval_seq[:1])         # the first frame, plain from the identity
    r0 = plain.read_back(V=False, flags=False)
    warm.set_node_params(r0["R"].reshape(-1, 9), r0["t"])
    warm.record_motion()
    res = ws.evaluate(plain, warm, net, eval_seq[1:], (sp, sw))
    sm = ws.summary(res)
    report("warm_start_gain_tiny", loss_first=losses[0][1], loss_last=losses[-1][1],
           rows=int(sum(f.shape[0] for f in Fs) * tiny.n_nodes), **sm)
    assert losses[-1][1] < 0.5 * losses[0][1]
    # the plain arm stops at its own final energy: every frame, within its budget
    assert sm["reached_plain"] == 1.0
    assert all(r["steps_plain"] <= tiny.n_gn for r in res)
    # the warm solve never starts above the plain one: a prediction that
    # raises the energy is rejected and the start restored
    for r in res:
        assert r["e_predicted"] <= r["e_start"] * (1 + 1e-6)
    net.close()
    plain.close()
    warm.close()
