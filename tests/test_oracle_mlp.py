"""The selector network's CPU reference gradient against central finite differences (no GPU)."""
import numpy as np

from oracle import mlp


def test_mlp_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    H = 7
    n = 6 * H + H + H * H + H + 2 * H + 2
    theta = rng.normal(0, 0.5, n)
    X = rng.normal(0, 1, (11, 6))
    T = rng.normal(0, 1, (11, 2))
    L, g = mlp.loss_and_grad(theta, H, X, T)
    assert abs(L - np.mean((mlp.forward(theta, H, X) - T) ** 2)) < 1e-14
    h = 1e-6
    for i in rng.choice(n, 40, replace=False):
        e = np.zeros(n)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, H, X, T)[0] - mlp.loss_and_grad(theta - e, H, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), i
