"""Pins of the FP64 reference network (oracle/mlp.py): each check compares it
with something other than itself -- finite differences, the erf form of the
GELU, closed forms of special cases and of Adam's first steps -- and planted
mistakes show that the checks bite."""
import math

import numpy as np
import pytest

from oracle import mlp


def rand_params(K, scale=0.5, seed=0):
    return np.random.default_rng(seed).normal(0.0, scale, mlp.nparams(K))


def test_gelu_identities():
    z = np.linspace(-6, 6, 1201)
    # tanh is odd, so g(z) - g(-z) = z exactly
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-14)
    assert mlp.gelu(0.0) == 0.0
    assert mlp.gelu_grad(0.0) == pytest.approx(0.5, abs=1e-15)
    # the tanh form approximates z Phi(z) (Phi the normal CDF, by math.erf)
    # to a few 1e-4
    exact = np.array([x * 0.5 * (1 + math.erf(x / math.sqrt(2))) for x in z])
    assert np.abs(mlp.gelu(z) - exact).max() < 1e-3
    # derivative against central differences
    h = 1e-5
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.abs(mlp.gelu_grad(z) - fd).max() < 1e-9
    # far tails: identity and zero
    assert mlp.gelu(12.0) == pytest.approx(12.0, rel=1e-15)
    assert abs(mlp.gelu(-12.0)) < 1e-30


def fd_grad(P, K, x, t, h=1e-6):
    g = np.empty_like(P)
    for i in range(P.size):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        g[i] = (mlp.loss(Pp, K, x, t) - mlp.loss(Pm, K, x, t)) / (2 * h)
    return g


def test_loss_grad_matches_finite_differences():
    K, B = 3, 7
    rng = np.random.default_rng(1)
    P = rand_params(K, seed=2)
    x = rng.uniform(-1, 1, B)
    t = rng.normal(0, 1, (B, K))
    L, g = mlp.loss_grad(P, K, x, t)
    assert L == pytest.approx(mlp.loss(P, K, x, t), rel=1e-15)
    fd = fd_grad(P, K, x, t)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(g).max()


def test_zero_output_weights_closed_form():
    """With W3 = 0 the output is b3, and only b3 gets a gradient:
    dL/db3_k = 2/(B K) sum_b (b3_k - t_bk)."""
    K, B = 4, 9
    rng = np.random.default_rng(3)
    P = rand_params(K, seed=4)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(P, K)
    W3[:] = 0.0
    x = rng.uniform(-1, 1, B)
    t = rng.normal(0, 1, (B, K))
    y, _ = mlp.forward(P, K, x)
    assert np.array_equal(y, np.broadcast_to(b3, (B, K)))
    L, g = mlp.loss_grad(P, K, x, t)
    assert L == pytest.approx(np.mean((b3[None, :] - t) ** 2), rel=1e-14)
    gW1, gb1, gW2, gb2, gW3, gb3 = mlp.unpack(g, K)
    assert not gW1.any() and not gb1.any() and not gW2.any() and not gb2.any()
    assert np.allclose(gb3, 2.0 / (B * K) * (b3[None, :] - t).sum(0), rtol=1e-14)
    # dW3 is the outer product of the output error with h2
    h2 = mlp.gelu(mlp.gelu(x[:, None] * W1 + b1) @ W2.T + b2)
    want = (2.0 / (B * K) * (b3[None, :] - t)).T @ h2
    assert np.allclose(gW3, want, rtol=1e-13, atol=1e-16)


def test_adam_first_steps_closed_form():
    """With bias correction the first step moves each parameter by
    lr g/(|g| + eps); under a constant gradient every later step does too."""
    rng = np.random.default_rng(5)
    P = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    want = lr * g / (np.abs(g) + eps)
    P1, m, v = mlp.adam(P, g, m, v, lr, b1, b2, eps, 1)
    assert np.allclose(P - P1, want, rtol=1e-12, atol=0)
    P2, m, v = mlp.adam(P1, g, m, v, lr, b1, b2, eps, 2)
    assert np.allclose(P1 - P2, want, rtol=1e-9, atol=0)


def mlp_variant(old: str, new: str):
    """A copy of oracle/mlp.py with one text replacement, loaded as its own
    module (the planted mistake lives only in the copy)."""
    import types
    src = open(mlp.__file__).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("mlp_variant")
    exec(compile(src.replace(old, new), "mlp_variant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("old,new", [
    # sign slip in the GELU derivative
    ("return 0.5 * (1.0 + t) + 0.5 * z", "return 0.5 * (1.0 + t) - 0.5 * z"),
    # lost factor 2 of d(y - t)^2/dy
    ("dy = 2.0 * (y - t) / (B * K)", "dy = 1.0 * (y - t) / (B * K)"),
    # W2 transposed in the backward pass
    ("dh1 = dz2 @ W2 ", "dh1 = dz2 @ W2.T "),
    # GELU derivative evaluated at the wrong layer's pre-activation
    ("dz1 = dh1 * gelu_grad(z1)", "dz1 = dh1 * gelu_grad(z2)"),
    # bias gradient averaged over the batch instead of summed
    ("db2 = dz2.sum(0)", "db2 = dz2.mean(0)"),
])
def test_planted_mistakes_are_caught(old, new):
    """Each plausible slip in the backward pass fails the finite-difference
    pin."""
    K, B = 2, 5
    rng = np.random.default_rng(6)
    P = rand_params(K, seed=7)
    x = rng.uniform(-1, 1, B)
    t = rng.normal(0, 1, (B, K))
    fd = fd_grad(P, K, x, t)
    good = mlp.loss_grad(P, K, x, t)[1]
    assert np.abs(good - fd).max() <= 1e-7 * np.abs(good).max()
    bad = mlp_variant(old, new)
    g = bad.loss_grad(P, K, x, t)[1]
    assert np.abs(g - fd).max() > 1e-3 * np.abs(fd).max()
