"""FP64 oracle for the learned cost model (test infrastructure only).

ORACLE: test infrastructure.  Only ``tests/`` may import it.  It shares no
code with the CUDA library.

The cost model is a multilayer perceptron with three hidden layers of 128
ReLU units and one linear output, trained with the mean squared error on the
(standardised) log of measured contraction time.  The paper estimates the
classical runtime as a FLOP count divided by the GPU's FLOP rate (Eq.
classical_runtime, §V) and reports that this consistently overestimates the
measured time (§VIII); the learned model replaces that ratio.

Parameter layout (flat vector, FP64 here, FP32 on the GPU):
    W1 [n_in x 128], b1 [128], W2 [128 x 128], b2 [128],
    W3 [128 x 128], b3 [128], W4 [128 x 1], b4 [1]
with Y = X W + b row-wise (rows of X are samples).

Everything below is the textbook chain rule for this network, written from
the definitions; :func:`finite_difference_grad` pins it independently.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 128
N_LAYERS = 4


def shapes(n_in: int):
    return [(n_in, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, 1), (1,)]


def n_params(n_in: int) -> int:
    return sum(int(np.prod(s)) for s in shapes(n_in))


def unpack(theta: np.ndarray, n_in: int):
    out, off = [], 0
    for s in shapes(n_in):
        k = int(np.prod(s))
        out.append(theta[off:off + k].reshape(s))
        off += k
    return out


def forward(theta: np.ndarray, X: np.ndarray):
    """Returns (prediction [n], activations list)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, X.shape[1])
    A0 = X
    Z1 = A0 @ W1 + b1
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ W2 + b2
    A2 = np.maximum(Z2, 0.0)
    Z3 = A2 @ W3 + b3
    A3 = np.maximum(Z3, 0.0)
    y = (A3 @ W4 + b4)[:, 0]
    return y, (A0, Z1, A1, Z2, A2, Z3, A3)


def loss(theta: np.ndarray, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(theta, X)
    return float(np.mean((y - t) ** 2))


def grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Gradient of the mean squared error by backpropagation."""
    n_in = X.shape[1]
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, n_in)
    y, (A0, Z1, A1, Z2, A2, Z3, A3) = forward(theta, X)
    B = X.shape[0]
    dy = (2.0 / B) * (y - t)[:, None]          # dL/dy
    gW4 = A3.T @ dy
    gb4 = dy.sum(axis=0)
    dA3 = dy @ W4.T
    dZ3 = dA3 * (Z3 > 0)
    gW3 = A2.T @ dZ3
    gb3 = dZ3.sum(axis=0)
    dA2 = dZ3 @ W3.T
    dZ2 = dA2 * (Z2 > 0)
    gW2 = A1.T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dA1 = dZ2 @ W2.T
    dZ1 = dA1 * (Z1 > 0)
    gW1 = A0.T @ dZ1
    gb1 = dZ1.sum(axis=0)
    return np.concatenate([g.reshape(-1) for g in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])


def finite_difference_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray, idx, h: float = 1e-6) -> np.ndarray:
    """Central differences of the loss at the parameter indices ``idx``."""
    out = np.empty(len(idx))
    for k, i in enumerate(idx):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        out[k] = (loss(tp, X, t) - loss(tm, X, t)) / (2 * h)
    return out


def adam_step(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) in FP64; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
