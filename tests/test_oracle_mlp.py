"""Pins of the oracle's MLP backprop (CPU): finite differences and closed forms."""
import numpy as np

from oracle import mlp


def setup(H=7, B=13, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.5, mlp.n_params(H))
    X = rng.normal(size=(B, 4))
    w = rng.normal(size=B)
    T = rng.normal(size=B)
    return p, X, w, T


def test_gradient_matches_central_differences():
    H = 7
    p, X, w, T = setup(H)
    g = mlp.grad(p, H, X, w, T)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(p + e, H, X, w, T) - mlp.loss(p - e, H, X, w, T)) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)


def test_output_layer_gradient_closed_form():
    # with the hidden layers fixed, L is quadratic in (w3, b3): dL/db3 = mean((w y - T) w)
    H = 5
    p, X, w, T = setup(H, seed=3)
    y, (h1, h2) = mlp.forward(p, H, X)
    g = mlp.grad(p, H, X, w, T)
    e = w * y - T
    assert np.isclose(g[-1], np.mean(e * w), rtol=1e-12)
    assert np.allclose(g[-1 - H:-1], (h2 * (e * w)[:, None]).mean(axis=0), rtol=1e-12)


def test_zero_loss_at_exact_fit():
    H = 4
    p, X, w, T = setup(H, seed=5)
    y, _ = mlp.forward(p, H, X)
    T = w * y
    assert mlp.loss(p, H, X, w, T) == 0.0
    assert np.all(mlp.grad(p, H, X, w, T) == 0.0)


def test_features_jacobi_limit():
    # the Jacobi factor -1/d is recoverable from the second input: x1 = 1/(16 d)
    f = mlp.features(np.array([3.0, -2.0, 1.5]), 1.0, 0.5, 0.1, 0.2)
    d = (np.array([3.0, -2.0, 1.5]) - 1.0) / 0.5
    assert np.allclose(f[:, 0], d) and np.allclose(f[:, 1], 1.0 / (16.0 * d))
    assert np.all(f[:, 2] == 0.1) and np.all(f[:, 3] == 0.2)
