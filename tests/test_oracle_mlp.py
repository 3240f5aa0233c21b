"""Pins for the oracle's warm-start network (oracle/mlp.py): gradients by
finite differences, a closed form when every ReLU is active, the first Adam
step, the rotation log against an independent library routine, and the
pooled node features on a hand-computed example."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import mlp


def _theta(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return rng.normal(scale=scale, size=mlp.N_PARAMS)


def test_parameter_count():
    assert mlp.N_PARAMS == 83974
    parts = mlp.unpack(np.arange(mlp.N_PARAMS, dtype=np.float64))
    assert [p.shape for p in parts] == [(64, 256), (256,), (256, 256), (256,), (256, 6), (6,)]
    assert np.array_equal(mlp.pack(parts), np.arange(mlp.N_PARAMS))


@pytest.mark.parametrize("scaled", [False, True])
def test_backward_matches_finite_differences(scaled):
    rng = np.random.default_rng(1)
    theta = _theta(2)
    x = rng.normal(size=(7, 64))
    t = rng.normal(size=(7, 6))
    s_out = rng.uniform(0.01, 3.0, size=6) if scaled else None
    y, cache = mlp.forward(theta, x, s_out)
    # keep every pre-activation away from the ReLU kink for the FD step
    assert min(np.abs(cache[1]).min(), np.abs(cache[3]).min()) > 1e-5
    L, dy = mlp.loss(y, t)
    g = mlp.backward(theta, cache, dy)
    idx = np.concatenate([rng.choice(64 * 256, 60, replace=False),                  # W1
                          64 * 256 + rng.choice(256, 10, replace=False),            # b1
                          64 * 256 + 256 + rng.choice(256 * 256, 60, replace=False),  # W2
                          mlp.N_PARAMS - 6 - 256 * 6 - 256 + rng.choice(256, 10, replace=False),  # b2
                          mlp.N_PARAMS - 6 - 256 * 6 + rng.choice(256 * 6, 30, replace=False),  # W3
                          mlp.N_PARAMS - 6 + np.arange(6)])                          # b3
    h = 1e-6
    for j in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (mlp.loss(mlp.forward(tp, x, s_out)[0], t)[0] - mlp.loss(mlp.forward(tm, x, s_out)[0], t)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(g[j])), (j, fd, g[j])


def test_all_active_network_is_the_composed_linear_map():
    """With positive biases large enough that every unit is active, the
    network is x -> x W1 W2 W3 + (b1 W2 W3 + b2 W3 + b3)."""
    rng = np.random.default_rng(3)
    W1 = rng.normal(scale=0.05, size=(64, 256))
    W2 = rng.normal(scale=0.05, size=(256, 256))
    W3 = rng.normal(scale=0.05, size=(256, 6))
    b1 = np.full(256, 50.0)
    b2 = np.full(256, 50.0) + np.abs(W2).sum(0) * 60.0
    b3 = rng.normal(size=6)
    theta = mlp.pack([W1, b1, W2, b2, W3, b3])
    x = rng.normal(size=(5, 64))
    y, cache = mlp.forward(theta, x)
    assert (cache[1] > 0).all() and (cache[3] > 0).all()
    A = np.linalg.multi_dot([W1, W2, W3])
    c = np.linalg.multi_dot([b1, W2, W3]) + b2 @ W3 + b3
    assert np.allclose(y, x @ A + c, rtol=1e-12, atol=1e-9)


def test_first_adam_step_moves_by_lr_times_sign():
    rng = np.random.default_rng(4)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    assert np.allclose(new - theta, -1e-3 * np.sign(g), rtol=1e-12, atol=0)


def test_rot_log_inverts_the_library_exponential():
    rng = np.random.default_rng(5)
    w = rng.normal(size=(200, 3))
    w *= (rng.uniform(1e-4, 3.0, size=200) / np.linalg.norm(w, axis=1))[:, None]
    R = Rotation.from_rotvec(w).as_matrix()
    assert np.allclose(mlp.rot_log(R), w, atol=1e-9)
    assert np.array_equal(mlp.rot_log(np.eye(3)[None]), np.zeros((1, 3)))


def test_node_features_hand_example():
    """Two nodes, three vertices: node 0 binds vertices 0 (w .75) and 1 (w .25),
    node 1 binds vertex 2 (w 1.0); one edge each way."""
    R = np.tile(np.eye(3), (2, 1, 1)).reshape(2, 9)
    t = np.array([[0.1, 0.2, 0.3], [0.0, 0.0, 0.0]])
    g = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    rhs = np.array([[1.0, -2.0, 0.0, 4.0, 0.0, 0.0], [0.0] * 6])
    diag = np.array([[2.0, 2.0, 1.0, 4.0, 1.0, 1.0], [0.0] * 6])
    r_photo = np.array([[1.0, -1.0, 2.0], [-3.0, 1.0, 2.0], [0.0, 0.0, 0.0]])
    r_sil = np.array([0.0, 2.0, 0.0])
    e = np.array([[0.5, 0.0, -1.0], [1.5, 2.0, 1.0], [0.0, 0.0, 0.0]])
    H = np.array([[1.0, 0.0, 0.0, 1.0, 0.0, 1.0], [3.0, 1.0, 0.0, 1.0, 0.0, 5.0], [0.0] * 6])
    flags = np.array([1, 1 | 2 | 4 | 8, 0], np.uint8)
    u_prev = np.array([[0.0, 0.0, 0.0, 1.0, 1.0, 1.0], [6.0, 0.0, 0.0, 0.0, 0.0, 0.0]])
    F = mlp.node_features(R, t, g, rhs, diag, np.array([0, 2, 3]), np.array([0, 1, 2]),
                          np.array([0.75, 0.25, 1.0]), r_photo, r_sil, e, H, flags, u_prev,
                          np.array([0, 1, 2]), np.array([1, 0]))
    f = F[0]
    assert np.array_equal(f[0:3], [0, 0, 0]) and np.allclose(f[3:6], [0.1, 0.2, 0.3])
    tau = 1e-6 * 4.0 + 1e-30
    assert np.allclose(f[18:24], rhs[0] / (diag[0] + tau))
    assert np.allclose(f[24:27], [0.75 * 1 + 0.25 * -3, 0.75 * -1 + 0.25 * 1, 2.0])
    assert np.allclose(f[27:30], [1.5, 1.0, 2.0])
    assert np.allclose(f[30:32], [0.5, 1.0])
    assert np.allclose(f[32:35], [0.75, 0.5, -0.5])
    assert np.allclose(f[35:38], [0.75, 0.5, 1.0])
    assert np.allclose(f[38:44], [1.5, 0.25, 0.0, 1.0, 0.0, 2.0])
    assert np.allclose(f[44:48], [1.0, 0.25, 0.25, 1.0])
    assert np.allclose(f[48:51], [1, 2, 3]) and np.allclose(f[51:57], u_prev[0])
    assert np.allclose(f[57:63], u_prev[1]) and f[63] == 1.0
    # node 1: its only vertex is inactive (zero residuals, no flags)
    assert np.allclose(F[1, 24:47], 0.0) and F[1, 47] == 1.0 and np.allclose(F[1, 57:63], u_prev[0])


def test_output_scale_multiplies_each_output():
    rng = np.random.default_rng(6)
    theta = _theta(7)
    x = rng.normal(size=(4, 64))
    s_out = np.array([0.5, 2.0, 1.0, 1e-3, 7.0, 1.0])
    y1, _ = mlp.forward(theta, x)
    y2, _ = mlp.forward(theta, x, s_out)
    assert np.allclose(y2, y1 * s_out, rtol=1e-14, atol=0)


def test_fit_scaling_normalises_the_training_rows():
    """After fitting, the normalised features have zero mean and unit
    population variance per column (the constant column and a constant
    feature excepted) and the scaled targets unit root mean square."""
    rng = np.random.default_rng(8)
    F = rng.normal(size=(500, 64)) * rng.uniform(1e-3, 50.0, size=64) + rng.normal(scale=20.0, size=64)
    F[:, 63] = 1.0
    F[:, 10] = 4.25                       # a constant feature
    T = rng.normal(size=(500, 6)) * np.array([0.02, 0.03, 0.01, 2e-3, 1e-3, 5e-3]) + 1e-3
    T[:, 5] = 0.0                         # an all-zero target column
    mu, sigma, s_out = mlp.fit_scaling(F, T)
    X = (F - mu) / sigma
    live = [j for j in range(63) if j != 10]
    assert np.allclose(X[:, live].mean(0), 0.0, atol=1e-9)     # rounding of a mean ~20 over sigma ~1e-3
    assert np.allclose(X[:, live].std(0), 1.0, rtol=1e-9)
    assert mu[63] == 0.0 and sigma[63] == 1.0 and np.all(X[:, 63] == 1.0)
    assert sigma[10] == 1.0 and np.all(X[:, 10] == 0.0)
    Ts = T[:, :5] / s_out[:5]
    assert np.allclose(np.sqrt((Ts * Ts).mean(0)), 1.0, rtol=1e-12)
    assert s_out[5] == 1.0


def test_node_motion_recovers_the_applied_rotation():
    """R_end = Exp(w) R_start (library exponential) gives back w; the
    translation part is the plain difference."""
    rng = np.random.default_rng(9)
    n = 50
    Rs = Rotation.from_rotvec(rng.normal(scale=0.8, size=(n, 3))).as_matrix()
    w = rng.normal(size=(n, 3))
    w *= (rng.uniform(1e-4, 2.5, size=n) / np.linalg.norm(w, axis=1))[:, None]
    Re = np.einsum("nij,njk->nik", Rotation.from_rotvec(w).as_matrix(), Rs)
    ts, te = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    u = mlp.node_motion(Rs.reshape(n, 9), ts, Re.reshape(n, 9), te)
    assert np.allclose(u[:, :3], w, atol=1e-9)
    assert np.array_equal(u[:, 3:], te - ts)
