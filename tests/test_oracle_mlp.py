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


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = _theta(2)
    x = rng.normal(size=(7, 64))
    t = rng.normal(size=(7, 6))
    y, cache = mlp.forward(theta, x)
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
        fd = (mlp.loss(mlp.forward(tp, x)[0], t)[0] - mlp.loss(mlp.forward(tm, x)[0], t)[0]) / (2 * h)
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
