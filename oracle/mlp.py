"""Oracle of the learned warm start (TEST INFRASTRUCTURE ONLY).

The paper has no network; the warm start is an addition of this library: a
per-vertex MLP predicts the correction r to the constant-velocity guess, and
the local-global iteration of a step starts from q0 = 2 x_t - x_{t-1} + r
instead of q_t (Alg. 1 starts from q_t). The converged result does not depend
on the start, so the network can only change iteration counts.

Everything here is the plain definition, in FP64:
  features   f_v = [x_t - x_{t-1}, x_t - X, log10(E_v / 1e5)], E_v the
             volume-weighted mean Young's modulus of the elements around v;
  network    4 dense layers 7 -> H -> H -> H -> 3, ReLU between layers, on
             normalised features (f - mean) / scale; output times oscale;
  loss       mean squared error over the batch and the 3 outputs, of the
             normalised output against the normalised target
             r* = x_{t+1} - (2 x_t - x_{t-1});
  gradient   backpropagation written out layer by layer;
  Adam       Kingma & Ba (2015), Algorithm 1, with bias correction;
  BF16       round-to-nearest-even of an FP32 value to 8 mantissa bits.
Parameter layout (one flat vector): W1 [H][7], b1 [H], W2 [H][H], b2 [H],
W3 [H][H], b3 [H], W4 [3][H], b4 [3].
"""
from __future__ import annotations

import numpy as np

N_IN, N_OUT = 7, 3


def n_params(H: int = 128) -> int:
    return H * N_IN + H + 2 * (H * H + H) + N_OUT * H + N_OUT


def unpack(theta: np.ndarray, H: int = 128):
    """Views (W1, b1, W2, b2, W3, b3, W4, b4) of the flat parameter vector."""
    shapes = [(H, N_IN), (H,), (H, H), (H,), (H, H), (H,), (N_OUT, H), (N_OUT,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    assert o == theta.size
    return out


def bf16_round(x) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), returned as
    FP32. Finite inputs only."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def vertex_log_stiffness(X, tets, E) -> np.ndarray:
    """log10(E_v / 1e5) with E_v the volume-weighted mean of E over the
    elements incident to v."""
    X = np.asarray(X, dtype=np.float64)
    tets = np.asarray(tets)
    D = X[tets[:, 1:]] - X[tets[:, :1]]
    V = np.abs(np.linalg.det(D)) / 6.0
    num = np.zeros(X.shape[0])
    den = np.zeros(X.shape[0])
    for a in range(4):
        np.add.at(num, tets[:, a], V * E)
        np.add.at(den, tets[:, a], V)
    return np.log10(num / den / 1e5)


def features(x_t, x_tm1, X, logE) -> np.ndarray:
    """Raw per-vertex features [x_t - x_{t-1}, x_t - X, log10(E_v/1e5)]."""
    return np.concatenate([x_t - x_tm1, x_t - X, np.asarray(logE)[:, None]], axis=1)


def target(x_tp1, x_t, x_tm1) -> np.ndarray:
    """Correction to the constant-velocity guess: x_{t+1} - (2 x_t - x_{t-1})."""
    return x_tp1 - (2.0 * x_t - x_tm1)


def forward(theta, feat_norm, H: int = 128, keep: bool = False):
    """Network output (normalised units) for normalised features [n, 7]."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(np.asarray(theta, dtype=np.float64), H)
    a0 = np.asarray(feat_norm, dtype=np.float64)
    z1 = a0 @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ W3.T + b3
    a3 = np.maximum(z3, 0.0)
    y = a3 @ W4.T + b4
    if keep:
        return y, (a0, z1, a1, z2, a2, z3, a3)
    return y


def loss(theta, feat_norm, targ_norm, H: int = 128) -> float:
    y = forward(theta, feat_norm, H)
    return float(np.mean((y - targ_norm) ** 2))


def grad(theta, feat_norm, targ_norm, H: int = 128):
    """(loss, dloss/dtheta) by backpropagation through the four layers."""
    theta = np.asarray(theta, dtype=np.float64)
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, H)
    y, (a0, z1, a1, z2, a2, z3, a3) = forward(theta, feat_norm, H, keep=True)
    n = y.shape[0]
    dy = 2.0 * (y - targ_norm) / (n * N_OUT)
    g = []
    dW4 = dy.T @ a3
    db4 = dy.sum(0)
    dz3 = (dy @ W4) * (z3 > 0)
    dW3 = dz3.T @ a2
    db3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * (z2 > 0)
    dW2 = dz2.T @ a1
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ a0
    db1 = dz1.sum(0)
    for t in (dW1, db1, dW2, db2, dW3, db3, dW4, db4):
        g.append(t.reshape(-1))
    return float(np.mean((y - targ_norm) ** 2)), np.concatenate(g)


class Adam:
    """Kingma & Ba (2015), Algorithm 1: first and second moment estimates with
    bias correction; theta <- theta - lr * m_hat / (sqrt(v_hat) + eps)."""

    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def warm_start(theta_bf16, norm, x_t, x_tm1, X, logE, pinned, H: int = 128):
    """q0 = 2 x_t - x_{t-1} + oscale * net((f - mean) / scale) on free
    vertices; pinned vertices at X. norm = (mean[7], scale[7], oscale[3])."""
    mean, scale, oscale = norm
    f = (features(x_t, x_tm1, X, logE) - mean) / scale
    r = forward(theta_bf16, f, H) * oscale
    q0 = 2.0 * x_t - x_tm1 + r
    q0[np.asarray(pinned, dtype=bool)] = X[np.asarray(pinned, dtype=bool)]
    return q0
