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
    for _ in range(prob.get("ep", 0)):
        yield "ep", o, 3, 0
        o += 3
    for _ in range(prob.get("ed", 0)):
        yield "ed", o, 3, 0
        o += 3


def _exp_gens():
    """Normalised extreme rays of the exponential cone K^e = cl{x1 >= x2 e^{x3/x2}, x2 > 0}
    (Sec. 2, cone (v)) and of its dual cl{-y3 e^{y2/y3} <= e y1, y3 < 0}."""
    rho = np.concatenate([-np.logspace(3, -3, 300), [0.0], np.linspace(-60, 60, 12001), np.logspace(-3, 2.5, 300)])
    GK = np.vstack([np.stack([np.exp(rho), np.ones_like(rho), rho], 1), [[1.0, 0, 0], [0, 0, -1.0]]])
    GD = np.vstack([np.stack([np.exp(rho - 1), -rho, -np.ones_like(rho)], 1), [[1.0, 0, 0], [0, 1.0, 0]]])
    return (GK / np.linalg.norm(GK, axis=1, keepdims=True), GD / np.linalg.norm(GD, axis=1, keepdims=True))


EXP_GK, EXP_GD = _exp_gens()


def in_exp(x, tol):
    """x in K^e, tested through duality: <x, g> >= -tol for every generator g of the dual cone."""
    return (EXP_GD @ np.asarray(x, float)).min() >= -tol


def in_exp_dual(y, tol):
    """y in (K^e)*: <y, g> >= -tol for every generator g of K^e (the definition of a dual cone)."""
    return (EXP_GK @ np.asarray(y, float)).min() >= -tol


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
        elif kind == "s":
            assert np.linalg.eigvalsh(svec_mat(blk, d)).min() >= -tol
        elif (kind == "ep") != dual:  # K^e: a primal block of K, or a dual block of K*
            assert in_exp(blk, tol), blk
        else:
            assert in_exp_dual(blk, tol), blk


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


def fista_logreg(Asmp, lam, iters=20000):
    """Independent FISTA for lam ||w||_1 + sum_i log(1 + exp(a_i^T w)) (FP64);
    returns (w, objective)."""
    Asmp = np.asarray(Asmp, float)
    L = 0.25 * np.linalg.norm(Asmp, 2) ** 2
    w = np.zeros(Asmp.shape[1])
    yv = w.copy()
    t = 1.0
    for _ in range(iters):
        z = Asmp @ yv
        grad = Asmp.T @ (0.5 * (1.0 + np.tanh(0.5 * z)))
        u = yv - grad / L
        wn = np.sign(u) * np.maximum(np.abs(u) - lam / L, 0.0)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        yv = wn + ((t - 1) / tn) * (wn - w)
        w, t = wn, tn
    obj = lam * np.abs(w).sum() + np.logaddexp(0.0, Asmp @ w).sum()
    return w, obj
