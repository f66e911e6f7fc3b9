"""Test-only helpers: dense restatements of the paper's definitions used as
independent pins for the oracle (never used by the product path)."""
from __future__ import annotations

import os

import numpy as np
import scipy.sparse as sp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dense_Q(A, b, c):
    """Q = [0 A^T c; -A 0 b; -c^T -b^T 0] of the HSDE (Sec. 3.1)."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A)
    m, n = A.shape
    N = n + m + 1
    Q = np.zeros((N, N))
    Q[:n, n:n + m] = A.T
    Q[:n, -1] = c
    Q[n:n + m, :n] = -A
    Q[n:n + m, -1] = b
    Q[-1, :n] = -c
    Q[-1, n:n + m] = -b
    return Q


def read_cases(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([[float(t) for t in part.split()] for part in line.split("|")])
    return rows


def in_soc(z, tol=1e-12):
    return np.linalg.norm(z[:-1]) <= z[-1] + tol * (1 + np.abs(z).max())


def cone_blocks(prob):
    """Yield (kind, start, length, order) for each cone block of s."""
    o = 0
    if prob.get("f", 0):
        yield "f", o, prob["f"], 0
        o += prob["f"]
    if prob.get("l", 0):
        yield "l", o, prob["l"], 0
        o += prob["l"]
    for k in prob.get("q", []):
        yield "q", o, k, 0
        o += k
    for d in prob.get("s", []):
        k = d * (d + 1) // 2
        yield "s", o, k, d
        o += k


def svec_mat(v, d):
    """mat of Sec. 2 written out independently of the oracle."""
    X = np.zeros((d, d))
    o = 0
    for j in range(d):
        for i in range(j, d):
            e = v[o] if i == j else v[o] / np.sqrt(2.0)
            X[i, j] = X[j, i] = e
            o += 1
    return X


def check_in_cone(prob, s, dual, tol):
    """Membership of s in K (dual=False) or K* (dual=True)."""
    for kind, o, k, d in cone_blocks(prob):
        blk = s[o:o + k]
        if kind == "f":
            if not dual:
                assert np.abs(blk).max() <= tol
        elif kind == "l":
            assert blk.min() >= -tol
        elif kind == "q":
            assert np.linalg.norm(blk[:-1]) <= blk[-1] + tol
        else:
            assert np.linalg.eigvalsh(svec_mat(blk, d)).min() >= -tol


def fista_lasso(F, g, mu, iters=20000):
    """Independent FISTA for 1/2||Fx-g||^2 + mu||x||_1 (dense, FP64)."""
    F = F.toarray() if sp.issparse(F) else np.asarray(F)
    L = np.linalg.norm(F, 2) ** 2
    x = np.zeros(F.shape[1])
    yv = x.copy()
    t = 1.0
    for _ in range(iters):
        grad = F.T @ (F @ yv - g)
        z = yv - grad / L
        xn = np.sign(z) * np.maximum(np.abs(z) - mu / L, 0.0)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        yv = xn + ((t - 1) / tn) * (xn - x)
        x, t = xn, tn
    return x
