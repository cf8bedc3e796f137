"""Pins of the FP64 network reference: central finite differences of its
loss, and closed forms of special parameter sets."""
import numpy as np
import pytest

from oracle import mlp


def rand_params(rng, scale=0.3):
    return rng.normal(0.0, scale, mlp.NPARAMS)


@pytest.mark.parametrize("under", [1.0, 4.0])
def test_gradient_matches_central_differences(under):
    rng = np.random.default_rng(17)
    p = rand_params(rng)
    x = rng.normal(0.0, 1.0, (24, 8))
    t = rng.normal(0.0, 1.0, 24)
    _, g = mlp.loss_and_grad(p, x, t, under)
    idx = np.concatenate([rng.choice(mlp.NPARAMS, 200, replace=False), [4800, 0, 575, 4735]])
    h = 1e-6
    for i in idx:
        q = p.copy(); q[i] += h
        lp, _ = mlp.loss_and_grad(q, x, t, under)
        q[i] -= 2 * h
        lm, _ = mlp.loss_and_grad(q, x, t, under)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_closed_forms():
    rng = np.random.default_rng(3)
    x = rng.normal(0.0, 1.0, (10, 8))
    t = rng.normal(0.0, 1.0, 10)
    # all weights zero except b3: y = b3, loss = mean (b3 - t)^2, only b3 has gradient
    p = np.zeros(mlp.NPARAMS); p[4800] = 0.7
    loss, g = mlp.loss_and_grad(p, x, t)
    assert np.isclose(loss, np.mean((0.7 - t) ** 2))
    assert np.isclose(g[4800], 2 * np.mean(0.7 - t))
    assert np.count_nonzero(g) == 1
    # the weighted loss weighs only the rows whose output is below the target
    loss4, g4 = mlp.loss_and_grad(p, x, t, under=4.0)
    w = np.where(0.7 < t, 4.0, 1.0)
    assert np.isclose(loss4, np.mean(w * (0.7 - t) ** 2))
    assert np.isclose(g4[4800], 2 * np.mean(w * (0.7 - t)))
    # identity-like path: W1 copies x0 to unit 0, W2 copies unit 0 to unit 0,
    # w3 reads unit 0: y = relu(relu(x0)) = relu(x0)
    W1 = np.zeros((8, 64)); W1[0, 0] = 1.0
    W2 = np.zeros((64, 64)); W2[0, 0] = 1.0
    w3 = np.zeros(64); w3[0] = 1.0
    p = mlp.pack(W1, np.zeros(64), W2, np.zeros(64), w3, 0.0)
    assert np.allclose(mlp.forward(p, x), np.maximum(x[:, 0], 0.0))


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159265, -0.1, 65504.0])
    r = mlp.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7   # tie to even, exact
    assert abs(r[3] - 3.140625) < 1e-12 and abs(r[4] + 0.10009765625) < 1e-12
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8)
