"""Pins of the MLP oracle: the backward pass against central finite
differences of its own loss (FP64), on a network small enough to perturb
every parameter; the Adam update against closed forms of its iterates derived
by hand from the definition (moving averages with bias correction)."""
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


def test_adam_first_step_is_normalised_gradient():
    # at t = 1 from m = v = 0 the bias corrections give mhat = g, vhat = g^2,
    # so the step is lr * g / (|g| + eps) whatever the betas
    theta = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.2, -4.0, 0.0, 1e-3])
    lr = 0.01
    t1, m1, v1 = M.adam_step(theta, g, np.zeros(4), np.zeros(4), 1, lr)
    np.testing.assert_allclose(t1, theta - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-16)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-13)
    assert t1[2] == 0.5  # a zero gradient leaves the parameter (and no NaN from 0 / eps)


def test_adam_constant_gradient_moves_linearly():
    # with a constant gradient the corrected moments are exactly g and g^2 at
    # every step (geometric sums: m_t = g (1 - b1^t), v_t = g^2 (1 - b2^t)),
    # so theta_t = theta_0 - t lr g / (|g| + eps)
    theta0 = np.array([0.3, -1.0, 2.0])
    g = np.array([0.5, -2.0, 1e-4])
    lr = 1e-3
    th, m, v = theta0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 41):
        th, m, v = M.adam_step(th, g, m, v, t, lr)
        np.testing.assert_allclose(m, g * (1 - 0.9 ** t), rtol=1e-13)
        np.testing.assert_allclose(v, g * g * (1 - 0.999 ** t), rtol=1e-12)
        np.testing.assert_allclose(th, theta0 - t * lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_adam_alternating_gradient_closed_form():
    # g_t = (-1)^(t+1) a: v_t = a^2 (1 - b2^t), so vhat = a^2, and
    # m_t = (1 - b1) a (-1)^(t+1) sum_{j<t} (-b1)^j = 0.1 a (-1)^(t+1) (1 - (-0.9)^t) / 1.9,
    # hence theta_t - theta_{t-1} = -lr mhat_t / (|a| + eps) with mhat_t = m_t / (1 - 0.9^t)
    a = np.array([0.7, -3.0])
    lr = 0.05
    th, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 25):
        g = a * (-1.0) ** (t + 1)
        prev = th
        th, m, v = M.adam_step(th, g, m, v, t, lr)
        m_closed = 0.1 * a * (-1.0) ** (t + 1) * (1 - (-0.9) ** t) / 1.9
        np.testing.assert_allclose(m, m_closed, rtol=1e-12)
        np.testing.assert_allclose(th - prev, -lr * (m_closed / (1 - 0.9 ** t)) / (np.abs(a) + 1e-8),
                                   rtol=1e-11, atol=1e-16)


def test_adam_wrong_bias_correction_is_caught():
    # planted mistake (in a copy of the oracle's step, on the CPU): dropping the
    # correction of v breaks the constant-gradient pin at t = 2
    def bad_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        return theta - lr * (m / (1 - beta1 ** t)) / (np.sqrt(v) + eps), m, v

    g = np.array([0.5])
    th, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    for t in (1, 2):
        th, m, v = bad_step(th, g, m, v, t, 1e-3)
    assert abs(th[0] - (-2e-3 * 0.5 / (0.5 + 1e-8))) > 1e-4
