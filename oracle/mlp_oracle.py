"""Plain FP64 numpy reference of the warm-start MLP (forward, loss, backward,
and the Adam update that trains it).

TEST INFRASTRUCTURE ONLY (tests and the benchmark's checks).  The paper has no
counterpart; the network follows include/superscs_mlp.h:
    xn = (x - in_mean) / in_std
    h1 = relu(xn W1^T + b1),  h2 = relu(h1 W2^T + b2),  y = h2 W3^T + b3
    loss = 0.5 * mean over batch and outputs of (y - (t - out_mean) / out_std)^2
Parameters are one flat vector in the order W1, b1, W2, b2, W3, b3 with each
W stored row-major (outputs x inputs).  The update is Adam as Kingma and Ba
publish it (ICLR 2015, Algorithm 1: exponential moving averages of the
gradient and of its square, each divided by its bias correction 1 - beta^t).
Pins: finite differences for the backward pass; hand-derived closed forms of
the Adam iterates (first step, constant and alternating gradients).
"""
from __future__ import annotations

import numpy as np


def unpack(theta, din, dh, dout):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    out = []
    for shape in ((dh, din), (dh,), (dh, dh), (dh,), (dout, dh), (dout,)):
        k = int(np.prod(shape))
        out.append(theta[o:o + k].reshape(shape))
        o += k
    assert o == theta.size
    return out


def loss_and_grad(theta, X, T, dims, norm=None):
    din, dh, dout = dims
    W1, b1, W2, b2, W3, b3 = unpack(theta, din, dh, dout)
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    if norm is None:
        norm = (np.zeros(din), np.ones(din), np.zeros(dout), np.ones(dout))
    im, isd, om, osd = (np.asarray(a, np.float64) for a in norm)
    xn = (X - im) / isd
    z1 = xn @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    y = h2 @ W3.T + b3
    tn = (T - om) / osd
    diff = y - tn
    B = X.shape[0]
    loss = 0.5 * np.mean(diff ** 2)
    dy = diff / (B * dout)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = (dy @ W3) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    gW1 = dh1.T @ xn
    gb1 = dh1.sum(0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad, y * osd + om


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Step t (t = 1, 2, ...) of Adam in FP64 (Kingma and Ba, Algorithm 1):
        m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g*g,
        theta <- theta - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
    Returns the new (theta, m, v); the inputs are not modified."""
    theta, g, m, v = (np.asarray(a, np.float64) for a in (theta, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
