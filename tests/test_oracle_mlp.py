"""Pins for the FP64 surrogate-network oracle (oracle/mlp.py).

The backward pass is checked against central finite differences of the loss
(a definition independent of the chain rule written in the oracle), the
first Adam step against its closed form (bias correction makes it
-lr * sign(g) up to eps), and a fit of a known smooth function shows that
forward, backward and Adam together minimise the loss.
"""
import numpy as np
import pytest

from oracle import mlp


@pytest.fixture
def net():
    K, H = 6, 16
    p = mlp.init_params(K, H, seed=3)
    for k in ("b1", "b2", "b3"):
        p[k] = np.random.default_rng(1).uniform(-0.1, 0.1, p[k].shape)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (9, K))
    t = rng.normal(size=9)
    return K, H, p, X, t


def test_backward_matches_central_differences(net):
    K, H, p, X, t = net
    g, L = mlp.backward(p, X, t)
    assert L == pytest.approx(mlp.loss(p, X, t), rel=1e-14)
    v = mlp.flatten(p)
    gv = mlp.flatten(g)
    h = 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(v.size, 60, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (mlp.loss(mlp.unflatten(vp, K, H), X, t) - mlp.loss(mlp.unflatten(vm, K, H), X, t)) / (2 * h)
        assert gv[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_first_adam_step_closed_form(net):
    K, H, p, X, t = net
    g, _ = mlp.backward(p, X, t)
    before = {k: v.copy() for k, v in p.items()}
    opt = mlp.Adam(p, lr=1e-2, eps=1e-12)
    opt.step(p, g)
    for k in p:
        # m_hat = g, v_hat = g^2 after bias correction: the step is -lr sign(g)
        expect = before[k] - 1e-2 * np.sign(g[k]) * (np.abs(g[k]) > 0)
        assert np.allclose(p[k], expect, atol=1e-9)


def test_fit_known_function():
    rng = np.random.default_rng(7)
    K, H = 4, 32
    X = rng.uniform(-1, 1, (512, K))
    t = np.sin(2 * X[:, 0]) + X[:, 1] ** 2 - 0.5 * X[:, 2] * X[:, 3]
    p = mlp.init_params(K, H, seed=1)
    opt = mlp.Adam(p, lr=3e-3)
    L0 = mlp.loss(p, X, t)
    for it in range(1500):
        idx = rng.choice(512, 64, replace=False)
        g, _ = mlp.backward(p, X[idx], t[idx])
        opt.step(p, g)
    assert mlp.loss(p, X, t) < 0.02 * L0


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie and rounds to even
    # (1.0); 1 + 3*2^-9 rounds up to 1 + 2^-7; integers up to 256 are exact
    assert mlp.to_bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.to_bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    assert np.array_equal(mlp.to_bf16(np.arange(257.0)), np.arange(257.0))
    x = np.random.default_rng(0).normal(size=1000)
    assert np.all(np.abs(mlp.to_bf16(x) - x) <= np.abs(x) * 2.0 ** -8)
