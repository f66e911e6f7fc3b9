"""Pins of the MLP oracle's backward pass: central finite differences of its
own loss (FP64), on a network small enough to perturb every parameter."""
import numpy as np

from oracle import mlp_oracle as M


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    dims = (5, 8, 4)
    n = 8 * 5 + 8 + 8 * 8 + 8 + 4 * 8 + 4
    theta = rng.standard_normal(n) * 0.5
    X = rng.standard_normal((6, 5))
    T = rng.standard_normal((6, 4))
    norm = (rng.standard_normal(5) * 0.1, rng.uniform(0.5, 2, 5), rng.standard_normal(4), rng.uniform(0.5, 2, 4))
    loss, g, _ = M.loss_and_grad(theta, X, T, dims, norm)
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (M.loss_and_grad(theta + e, X, T, dims, norm)[0] - M.loss_and_grad(theta - e, X, T, dims, norm)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-8)


def test_forward_output_units():
    rng = np.random.default_rng(1)
    dims = (3, 8, 2)
    theta = np.zeros(8 * 3 + 8 + 64 + 8 + 16 + 2)
    theta[-2:] = [1.0, -2.0]  # b3
    X = rng.standard_normal((4, 3))
    norm = (np.zeros(3), np.ones(3), np.array([10.0, 20.0]), np.array([2.0, 3.0]))
    _, _, y = M.loss_and_grad(theta, X, np.zeros((4, 2)), dims, norm)
    np.testing.assert_allclose(y, np.tile([10.0 + 2.0, 20.0 - 6.0], (4, 1)))
