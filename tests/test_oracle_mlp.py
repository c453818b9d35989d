"""Pins of the warm-start oracle (oracle/mlp.py) against facts that do not come
from the oracle itself: exact BF16 roundings, central finite differences of
the loss, Adam's closed-form first steps, hand-computed vertex stiffness, and
the constant-velocity special cases."""
import struct

import numpy as np
import pytest

from oracle import mlp


def f32(bits: int) -> float:
    return struct.unpack("<f", struct.pack("<I", bits))[0]


@pytest.mark.parametrize("inp, out", [
    (0x3F800000, 0x3F800000),   # 1.0 is representable
    (0x3F808000, 0x3F800000),   # 1 + 2^-8: tie, mantissa of 1.0 is even -> down
    (0x3F818000, 0x3F820000),   # 1 + 3 * 2^-8: tie, odd lower neighbour -> up
    (0x3F812345, 0x3F810000),   # below half -> down
    (0x3F81C000, 0x3F820000),   # above half -> up
    (0xC0200000, 0xC0200000),   # -2.5 representable
    (0xBF80FFFF, 0xBF810000),   # negative, above half -> away from zero
    (0x7F7FFFFF, 0x7F800000),   # largest float rounds to +inf in BF16
])
def test_bf16_round_known_patterns(inp, out):
    got = mlp.bf16_round(np.array([f32(inp)], dtype=np.float32))[0]
    assert struct.unpack("<I", struct.pack("<f", got))[0] == out


def _tiny(H=5, n=9, seed=0):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mlp.n_params(H)) * 0.7
    x = rng.standard_normal((n, mlp.N_IN))
    t = rng.standard_normal((n, mlp.N_OUT))
    return theta, x, t


def test_gradient_matches_central_differences():
    H = 5
    theta, x, t = _tiny(H)
    L, g = mlp.grad(theta, x, t, H)
    assert abs(L - mlp.loss(theta, x, t, H)) <= 1e-15 * max(1.0, L)
    h = 1e-6
    fd = np.zeros_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        fd[i] = (mlp.loss(theta + e, x, t, H) - mlp.loss(theta - e, x, t, H)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_layout_and_parameter_count():
    assert mlp.n_params(128) == 34435
    parts = mlp.unpack(np.arange(mlp.n_params(4), dtype=np.float64), 4)
    assert [p.shape for p in parts] == [(4, 7), (4,), (4, 4), (4,), (4, 4), (4,), (3, 4), (3,)]
    assert parts[0][0, 0] == 0 and parts[-1][-1] == mlp.n_params(4) - 1


def test_output_layer_only_network():
    # every hidden layer is dead (bias -1, zero weights): the output is b4
    H = 4
    theta = np.zeros(mlp.n_params(H))
    W1, b1, W2, b2, W3, b3, W4, b4 = mlp.unpack(theta, H)
    b1[:] = -1.0
    b4[:] = [0.5, -2.0, 3.0]
    y = mlp.forward(theta, np.random.default_rng(1).standard_normal((6, 7)), H)
    assert np.array_equal(y, np.tile([0.5, -2.0, 3.0], (6, 1)))


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(2)
    th0 = rng.standard_normal(11)
    g = rng.standard_normal(11)
    opt = mlp.Adam(11, lr=1e-2)
    th1 = opt.step(th0, g)
    # m_hat = g and v_hat = g^2 after bias correction
    assert np.allclose(th1, th0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    th2 = opt.step(th1, g)
    assert np.allclose(th2, th0 - 2e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_vertex_log_stiffness_hand_example():
    # two tets sharing the face (1,2,3): volumes 1/6 and 2/6
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 2]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3], [4, 1, 3, 2]])
    V = np.abs(np.linalg.det(X[tets[:, 1:]] - X[tets[:, :1]])) / 6
    assert np.isclose(V[0], 1 / 6)
    E = np.array([1e5, 1e7])
    le = mlp.vertex_log_stiffness(X, tets, E)
    shared = (V[0] * 1e5 + V[1] * 1e7) / (V[0] + V[1])
    assert np.isclose(le[0], 0.0)
    assert np.isclose(le[4], 2.0)
    assert np.allclose(le[1:4], np.log10(shared / 1e5))


def test_constant_velocity_motion_has_zero_target_and_zero_net_gives_extrapolation():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((10, 3))
    v = rng.standard_normal((10, 3))
    h = 0.01
    x0, x1, x2 = X + 0 * h * v, X + h * v, X + 2 * h * v
    assert np.allclose(mlp.target(x2, x1, x0), 0.0, atol=1e-15)
    pinned = np.zeros(10, dtype=np.uint8)
    pinned[:2] = 1
    norm = (np.zeros(7), np.ones(7), np.ones(3))
    q0 = mlp.warm_start(np.zeros(mlp.n_params(8)), norm, x1, x0, X, np.zeros(10), pinned, H=8)
    assert np.allclose(q0[2:], x2[2:], atol=1e-15)
    assert np.array_equal(q0[:2], X[:2])
