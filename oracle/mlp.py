"""FP64 reference of the rate surrogate's network and of its training step.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests, the
smoke check and the CPU leg of the benchmark may call it; the library never
does.

The paper evaluates the ADK rate of Eq. 1 directly.  The surrogate is a
small network that maps the field magnitude to the logarithms of all Z rates
of a species at once:

    h1 = g(W1 x + b1)            W1, b1: H       (x a scalar input)
    h2 = g(W2 h1 + b2)           W2: H x H, b2: H
    y  = W3 h2 + b3              W3: K x H, b3: K

with H = 64 and the GELU in its tanh form

    g(z) = z/2 (1 + tanh(c (z + 0.044715 z^3))),   c = sqrt(2/pi).

Training minimizes the mean squared error over a batch of B inputs and the
K outputs, L = (1/(B K)) sum_b sum_k (y_bk - t_bk)^2, with Adam.

Parameters travel as one flat array in the order W1, b1, W2 (row o holds the
weights into unit o), b2, W3 (row k), b3: H + H + H*H + H + K*H + K values.

Everything here is the textbook definition written out with numpy in
double precision: the forward pass, the chain rule for the gradient, and one
Adam update (Kingma & Ba, Algorithm 1).  Pins: tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def nparams(K: int) -> int:
    return H + H + H * H + H + K * H + K


def unpack(P: np.ndarray, K: int):
    """Views (W1, b1, W2, b2, W3, b3) into the flat parameter array."""
    P = np.asarray(P, dtype=np.float64)
    if P.size != nparams(K):
        raise ValueError(f"expected {nparams(K)} parameters, got {P.size}")
    o = 0
    out = []
    for shape in ((H,), (H,), (H, H), (H,), (K, H), (K,)):
        n = int(np.prod(shape))
        out.append(P[o:o + n].reshape(shape))
        o += n
    return tuple(out)


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    """d g / d z by the product and chain rules."""
    z = np.asarray(z, dtype=np.float64)
    u = GELU_C * (z + GELU_A * z ** 3)
    t = np.tanh(u)
    du = GELU_C * (1.0 + 3.0 * GELU_A * z * z)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def forward(P, K: int, x):
    """Outputs y (B, K) for inputs x (B,), and the intermediate values."""
    W1, b1, W2, b2, W3, b3 = unpack(P, K)
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    z1 = x[:, None] * W1[None, :] + b1[None, :]
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2[None, :]
    h2 = gelu(z2)
    y = h2 @ W3.T + b3[None, :]
    return y, (x, z1, h1, z2, h2)


def loss(P, K: int, x, t) -> float:
    y, _ = forward(P, K, x)
    t = np.asarray(t, dtype=np.float64).reshape(y.shape)
    return float(np.mean((y - t) ** 2))


def loss_grad(P, K: int, x, t):
    """(L, dL/dP) with dL/dP in the flat parameter layout."""
    W1, b1, W2, b2, W3, b3 = unpack(P, K)
    y, (x, z1, h1, z2, h2) = forward(P, K, x)
    t = np.asarray(t, dtype=np.float64).reshape(y.shape)
    B = y.shape[0]
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / (B * K)            # dL/dy
    dW3 = dy.T @ h2                          # (K, H)
    db3 = dy.sum(0)
    dh2 = dy @ W3                            # (B, H)
    dz2 = dh2 * gelu_grad(z2)
    dW2 = dz2.T @ h1                         # (H, H)
    db2 = dz2.sum(0)
    dh1 = dz2 @ W2                           # (B, H)
    dz1 = dh1 * gelu_grad(z1)
    dW1 = (dz1 * x[:, None]).sum(0)
    db1 = dz1.sum(0)
    g = np.concatenate([dW1, db1, dW2.reshape(-1), db2, dW3.reshape(-1), db3])
    return L, g


def adam(P, g, m, v, lr: float, beta1: float, beta2: float, eps: float, t: int):
    """One Adam update (step t >= 1, bias-corrected moments).  Returns new
    (P, m, v)."""
    P = np.asarray(P, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return P - lr * mhat / (np.sqrt(vhat) + eps), m, v
