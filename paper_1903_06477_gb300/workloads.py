"""Seeded synthetic problem generators shared by the tests and the benchmark.

This module only *builds* problems (data A, b, c and the cone list, plus the
planted solution where there is one).  It contains none of the solver's
arithmetic, so both the FP64 oracle and the CUDA path can be fed from it.

Every problem is a dict with
    A  : scipy.sparse.csr_matrix (m x n), rows ordered [f | l | q... | s...]
    b, c : float64 arrays
    f, l : ints;  q, s : lists of cone dimensions (SOC dims; PSD orders)
plus optional planted ``xstar``, ``ystar``, ``sstar`` and ``meta``.

Recipes (the paper measures on self-generated random families, Sec. 5; the
shapes below follow those families and the workload sizes of the benchmark):
  lasso()          l1-regularised least squares in epigraph form (Sec. 5.3)
  planted()        random sparse cone program with a planted primal-dual pair
  planted_sdp()    planted SDP blocks plus orthant rows
  portfolio()      long-only mean-risk portfolio SOCP
  infeasible() / unbounded()   planted certificates (Sec. 3, theorems of the alternative)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def _csr(rows, cols, vals, m, n):
    A = sp.csr_matrix((np.asarray(vals, np.float64), (np.asarray(rows), np.asarray(cols))), shape=(m, n))
    A.sum_duplicates()
    A.sort_indices()
    return A


def random_pattern(rng, m, n, nnz_target):
    """Uniform random sparsity pattern with about nnz_target distinct entries,
    N(0,1) values, returned in CSR (row-major sorted) order."""
    total = m * n
    k = int(min(total, nnz_target))
    if k == 0:
        return sp.csr_matrix((m, n))
    if total <= 4 * k:
        lin = rng.choice(total, size=k, replace=False)
    else:
        lin = np.unique(rng.integers(0, total, size=int(k * 1.02) + 16, dtype=np.int64))
        if lin.size > k:
            lin = np.sort(rng.choice(lin, size=k, replace=False))
    lin = np.sort(lin)
    rows, cols = lin // n, lin % n
    vals = rng.standard_normal(lin.size)
    indptr = np.zeros(m + 1, np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return sp.csr_matrix((vals, cols.astype(np.int32), indptr), shape=(m, n))


def lasso(seed=0, p=60, nvar=120, density=0.1, k_nz=12, noise=0.01, mu_frac=0.1, F=None, g=None):
    """min 1/2 ||F x - g||^2 + mu ||x||_1 as a cone program.

    Variables (x in R^nvar, t in R^nvar, r); c = (0, mu 1, 1).
    Orthant rows: t - x >= 0, t + x >= 0.  One SOC (t last):
    (sqrt2 (F x - g), r - 1, r + 1), which encodes 1/2 ||F x - g||^2 <= r.
    Default: F 60 x 120 at 10% density, N(0, 1/60) values, planted x with 12
    N(0,1) nonzeros, g = F x + 0.01 N(0,1), mu = 0.1 ||F^T g||_inf.
    """
    rng = np.random.default_rng(seed)
    if F is None:
        Fd = sp.random(p, nvar, density=density, random_state=rng, format="csr",
                       data_rvs=lambda k: rng.standard_normal(k) / math.sqrt(p))
    else:
        Fd = sp.csr_matrix(F)
        p, nvar = Fd.shape
    if g is None:
        xt = np.zeros(nvar)
        idx = rng.choice(nvar, size=min(k_nz, nvar), replace=False)
        xt[idx] = rng.standard_normal(idx.size)
        g = Fd @ xt + noise * rng.standard_normal(p)
    else:
        xt = None
    mu = mu_frac * np.max(np.abs(Fd.T @ g))
    n = 2 * nvar + 1
    I = sp.identity(nvar, format="csr")
    Z = sp.csr_matrix((nvar, 1))
    rows_l1 = sp.hstack([I, -I, Z])
    rows_l2 = sp.hstack([-I, -I, Z])
    er = sp.csr_matrix(([-1.0], ([0], [2 * nvar])), shape=(1, n))
    soc_F = sp.hstack([-math.sqrt(2.0) * Fd, sp.csr_matrix((p, nvar)), sp.csr_matrix((p, 1))])
    A = sp.vstack([rows_l1, rows_l2, soc_F, er, er]).tocsr()
    A.sort_indices()
    b = np.concatenate([np.zeros(2 * nvar), -math.sqrt(2.0) * g, [-1.0, 1.0]])
    c = np.concatenate([np.zeros(nvar), mu * np.ones(nvar), [1.0]])
    return dict(A=A, b=b, c=c, f=0, l=2 * nvar, q=[p + 2], s=[],
                meta=dict(F=Fd, g=np.asarray(g), mu=mu, xtrue=xt, nvar=nvar))


def _unit(rng, k):
    v = rng.standard_normal(k)
    nv = np.linalg.norm(v)
    return v / nv if nv > 0 else np.eye(k)[0]


def _svec(X):
    d = X.shape[0]
    out = np.empty(d * (d + 1) // 2)
    o = 0
    for j in range(d):
        col = X[j:, j].copy()
        col[1:] *= math.sqrt(2.0)
        out[o:o + d - j] = col
        o += d - j
    return out


def _exp_pair(rng, case):
    """A complementary pair (x in K^e, z in (K^e)*) of the exponential cone
    K^e = cl{x1 >= x2 exp(x3/x2), x2 > 0} (Sec. 2, cone (v)): case 0 x
    interior, z = 0; case 1 x = 0, z interior; case 2 both on the boundary,
    x = c (e^rho, 1, rho) and z = lam (1, -e^rho (1 - rho), -e^rho), <x, z> = 0."""
    x, z = np.zeros(3), np.zeros(3)
    if case == 0:
        x2, x3 = rng.uniform(0.5, 1.5), rng.standard_normal()
        x[:] = (x2 * np.exp(x3 / x2) + rng.uniform(0.5, 1.5), x2, x3)
    elif case == 1:
        z3, z2 = -rng.uniform(0.5, 1.5), rng.standard_normal()
        z[:] = (-z3 * np.exp(z2 / z3) / np.e + rng.uniform(0.5, 1.5), z2, z3)
    else:
        rho, cc, lam = rng.uniform(-2, 2), rng.uniform(0.5, 1.5), rng.uniform(0.5, 1.5)
        x[:] = cc * np.array([np.exp(rho), 1.0, rho])
        z[:] = lam * np.array([1.0, -np.exp(rho) * (1 - rho), -np.exp(rho)])
    return x, z


def planted(seed=0, n=200, l=200, soc=(), psd=(), f=0, nnz=None, density=None, psd_rank=None, ep=0, ed=0):
    """Random sparse cone program with a planted strictly complementary
    primal-dual optimum (x*, y*, s*); b = A x* + s*, c = -A^T y*.

    Orthant rows: with prob 1/2 s ~ U(0.1,1), y = 0, else y ~ U(0.1,1), s = 0.
    SOC of dim k (t last), u uniform on the unit sphere of R^{k-1}, a, beta
    ~ U(0.5,1.5), cycling over three cases: s = a(u,1), y = 0;  y = beta(-u,1),
    s = 0;  s = a(u,1), y = beta(-u,1).  PSD of order d: V from the QR of a
    Gaussian, S = V diag(lam_1..lam_k, 0..) V^T, Y = V diag(0.., lam_{k+1}..) V^T
    with lam ~ U(0.5, 2) and k ~ U{d/4..3d/4}.  Zero-cone rows: s = 0, y ~ N(0,1).
    Exponential cones (ep primal blocks of K^e, then ed blocks of its dual),
    cycling over the three complementary cases of _exp_pair (for a dual
    block the roles of s and y swap).
    A has N(0,1) values at uniform random positions.
    """
    rng = np.random.default_rng(seed)
    soc, psd = list(soc), list(psd)
    m = f + l + sum(soc) + sum(d * (d + 1) // 2 for d in psd) + 3 * (ep + ed)
    if nnz is None:
        nnz = int(round((density if density is not None else 0.05) * m * n))
    A = random_pattern(rng, m, n, nnz)
    xs = rng.standard_normal(n)
    s = np.zeros(m)
    y = np.zeros(m)
    o = 0
    y[o:o + f] = rng.standard_normal(f)
    o += f
    pick = rng.random(l) < 0.5
    sv = rng.uniform(0.1, 1.0, l)
    yv = rng.uniform(0.1, 1.0, l)
    s[o:o + l] = np.where(pick, sv, 0.0)
    y[o:o + l] = np.where(pick, 0.0, yv)
    o += l
    for i, k in enumerate(soc):
        if k == 1:
            if i % 2 == 0:
                s[o] = rng.uniform(0.5, 1.5)
            else:
                y[o] = rng.uniform(0.5, 1.5)
        else:
            u = _unit(rng, k - 1)
            a, be = rng.uniform(0.5, 1.5, 2)
            case = i % 3
            if case in (0, 2):
                s[o:o + k - 1] = a * u
                s[o + k - 1] = a
            if case in (1, 2):
                y[o:o + k - 1] = -be * u
                y[o + k - 1] = be
        o += k
    for d in psd:
        G = rng.standard_normal((d, d))
        V, _ = np.linalg.qr(G)
        lo, hi = (d // 4, (3 * d) // 4) if psd_rank is None else (psd_rank, psd_rank)
        ks = int(rng.integers(max(lo, 0), hi + 1))
        lam = rng.uniform(0.5, 2.0, d)
        ls = np.where(np.arange(d) < ks, lam, 0.0)
        ly = np.where(np.arange(d) >= ks, lam, 0.0)
        S = (V * ls) @ V.T
        Y = (V * ly) @ V.T
        k = d * (d + 1) // 2
        s[o:o + k] = _svec(S)
        y[o:o + k] = _svec(Y)
        o += k
    for i in range(ep + ed):
        xk, zk = _exp_pair(rng, i % 3)
        if i < ep:
            s[o:o + 3], y[o:o + 3] = xk, zk
        else:
            s[o:o + 3], y[o:o + 3] = zk, xk
        o += 3
    assert o == m
    b = A @ xs + s
    c = -(A.T @ y)
    return dict(A=A, b=b, c=c, f=f, l=l, q=soc, s=psd, ep=ep, ed=ed, xstar=xs, ystar=y, sstar=s)


def c2_planted(seed=0, scale=1.0):
    """Large planted sparse program: n = 100k, m = 200k (100k orthant rows plus
    2000 SOCs of dim 50), A at 0.05% density (1e7 nonzeros).  ``scale`` shrinks
    n, the orthant block and the SOC count together, keeping ~50 nnz per row."""
    n = max(10, int(round(100_000 * scale)))
    l = max(10, int(round(100_000 * scale)))
    nq = max(1, int(round(2000 * scale)))
    m = l + 50 * nq
    nnz = int(round(50 * m))
    return planted(seed, n=n, l=l, soc=[50] * nq, nnz=nnz)


def c3_planted_sdp(seed=0, nblk=512, d=64, l=50_000, n=20_000, nnz=1_000_000):
    """Planted SDP: nblk PSD blocks of order d plus l orthant rows, A with
    about nnz N(0,1) entries at uniform random positions."""
    return planted(seed, n=n, l=l, psd=[d] * nblk, nnz=nnz)


def portfolio(seed=0, k=None, gamma=1.0):
    """Long-only mean-risk portfolio SOCP with k assets and rank k//10 factors:
    min -mu^T w + gamma t  s.t.  1^T w = 1,  w >= 0,  (F^T w, D^{1/2} w, t) in SOC.
    k ~ U{20..400}, F ~ N(0, 1/k), D = diag U[0.01, 0.1], mu ~ N(0.05, 0.02)."""
    rng = np.random.default_rng(seed)
    if k is None:
        k = int(rng.integers(20, 401))
    r = max(1, k // 10)
    F = rng.standard_normal((k, r)) / math.sqrt(k)
    Dg = rng.uniform(0.01, 0.1, k)
    mu = rng.normal(0.05, 0.02, k)
    n = k + 1
    w = np.arange(k)
    rows = np.concatenate([np.zeros(k, np.int64),              # zero cone: 1^T w = 1
                           1 + w,                               # orthant: s = w
                           (k + 1) + np.repeat(np.arange(r), k),  # SOC: F^T w
                           (k + 1 + r) + w,                     # SOC: D^{1/2} w
                           [2 * k + r + 1]])                    # SOC: t (last)
    cols = np.concatenate([w, w, np.tile(w, r), w, [k]])
    vals = np.concatenate([np.ones(k), -np.ones(k), -F.T.ravel(), -np.sqrt(Dg), [-1.0]])
    m = 2 * k + r + 2
    A = _csr(rows, cols, vals, m, n)
    b = np.zeros(m)
    b[0] = 1.0
    c = np.concatenate([-mu, [gamma]])
    return dict(A=A, b=b, c=c, f=1, l=k, q=[r + k + 1], s=[], meta=dict(k=k, r=r))


def c4_portfolios(count=4096, seed0=1000):
    """The batched family: independent portfolio SOCPs with k ~ U{20..400}."""
    return [portfolio(seed=seed0 + i) for i in range(count)]


def infeasible(seed=0, n=200, l=200, soc=(10,) * 4, nnz=None):
    """Planted primal-infeasible program: the first two orthant rows are a and
    -a with b_1 + b_2 = -1, so y = e_1 + e_2 certifies infeasibility."""
    P = planted(seed, n=n, l=l, soc=soc, nnz=nnz)
    rng = np.random.default_rng(seed + 7919)
    A = P["A"].tolil()
    a = rng.standard_normal(n) * (rng.random(n) < 0.1)
    A[0, :] = a
    A[1, :] = -a
    A = A.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    b = P["b"].copy()
    b[0] = 0.3
    b[1] = -1.3
    return dict(A=A, b=b, c=P["c"], f=0, l=l, q=list(soc), s=[], ycert=np.eye(A.shape[0])[0] + np.eye(A.shape[0])[1])


def unbounded(seed=0, n=200, l=200, soc=(10,) * 4, nnz=None):
    """Planted dual-infeasible (unbounded) program: column 0 is replaced by
    one with entries <= 0 in orthant rows only and c_0 = -1, so x = e_0 with
    s = -A e_0 in K certifies unboundedness (a planted feasible x* keeps the
    primal feasible)."""
    P = planted(seed, n=n, l=l, soc=soc, nnz=nnz)
    rng = np.random.default_rng(seed + 104729)
    A = P["A"].tolil()
    m = A.shape[0]
    col = np.zeros(m)
    sel = rng.random(l) < 0.2
    col[:l] = -np.abs(rng.standard_normal(l)) * sel
    A[:, 0] = col.reshape(-1, 1)
    A = A.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    xs = P["xstar"].copy()
    b = A @ xs + P["sstar"]
    c = P["c"].copy()
    c[0] = -1.0
    return dict(A=A, b=b, c=c, f=0, l=l, q=list(soc), s=[], xcert=np.eye(n)[0])


def lasso_family_matrix(seed=0, p=2000, nvar=5000, density=0.01):
    """Fixed F of the parametric LASSO family: p x nvar at the given density
    with N(0, 1/p) values."""
    rng = np.random.default_rng(seed)
    return sp.random(p, nvar, density=density, random_state=rng, format="csr",
                     data_rvs=lambda k: rng.standard_normal(k) / math.sqrt(p))


def lasso_family_rhs(F, seed, frac_nz=0.05, noise=0.01):
    """One instance parameter g = F x + 0.01 N(0,1) with x 5% sparse N(0,1)."""
    rng = np.random.default_rng(seed)
    nvar = F.shape[1]
    x = np.zeros(nvar)
    k = max(1, int(round(frac_nz * nvar)))
    idx = rng.choice(nvar, size=k, replace=False)
    x[idx] = rng.standard_normal(k)
    return F @ x + noise * rng.standard_normal(F.shape[0])


def lasso_family_bc(F, g, mu_frac=0.1):
    """b and c of the epigraph LASSO cone program (same layout as lasso())
    for the design F and parameter g; mu = mu_frac ||F^T g||_inf."""
    p, nvar = F.shape
    mu = mu_frac * np.max(np.abs(F.T @ g))
    b = np.concatenate([np.zeros(2 * nvar), -math.sqrt(2.0) * np.asarray(g, np.float64), [-1.0, 1.0]])
    c = np.concatenate([np.zeros(nvar), mu * np.ones(nvar), [1.0]])
    return b, c


def lasso_family_rhs_smooth(F, seed, base_seed=0, frac_nz=0.05, rel=0.1, noise=0.01):
    """A smoothly varying member of the LASSO family: a fixed sparse x_base
    (frac_nz of the entries N(0,1), from base_seed) scaled entrywise by
    (1 + rel N(0,1)) per instance, g = F x + noise N(0,1)."""
    nvar = F.shape[1]
    rb = np.random.default_rng(base_seed)
    xb = np.zeros(nvar)
    k = max(1, int(round(frac_nz * nvar)))
    idx = rb.choice(nvar, size=k, replace=False)
    xb[idx] = rb.standard_normal(k)
    rng = np.random.default_rng(seed)
    x = xb * (1.0 + rel * rng.standard_normal(nvar))
    return F @ x + noise * rng.standard_normal(F.shape[0])


def logreg(seed=0, p=100, q=120, lam=10.0, density=1.0, frac_nz=0.1):
    """Sparse l1-regularised logistic regression (Sec. 5.4) as a conic program
    with exponential cones.  Reading of the printed objective (its sign and
    indices are garbled): minimise lam ||w||_1 + sum_i log(1 + exp(a_i^T w)),
    with a_i = -y_i x_i (labels folded into the samples).  Data: features x_i
    with N(0,1) entries at `density`, a planted w0 with frac_nz N(0,1)
    nonzeros, labels y_i = sign(x_i^T w0 + 0.1 N(0,1)).

    Variables (w, t, u, v1, v2) of sizes (p, p, q, q, q); objective
    lam sum t + sum u.  Orthant rows: t - w >= 0, t + w >= 0, 1 - v1 - v2 >= 0;
    per sample two exponential cones (x1 >= x2 exp(x3/x2)):
    (v1_i, 1, a_i^T w - u_i) and (v2_i, 1, -u_i), which together say
    exp(a_i^T w - u_i) + exp(-u_i) <= 1, i.e. u_i >= log(1 + exp(a_i^T w))."""
    rng = np.random.default_rng(seed)
    if density >= 1.0:
        X = rng.standard_normal((q, p))
    else:
        X = (rng.random((q, p)) < density) * rng.standard_normal((q, p))
    w0 = np.zeros(p)
    nz = rng.choice(p, max(1, int(round(frac_nz * p))), replace=False)
    w0[nz] = rng.standard_normal(len(nz))
    lab = np.sign(X @ w0 + 0.1 * rng.standard_normal(q))
    lab[lab == 0] = 1.0
    Asmp = -lab[:, None] * X
    n = 2 * p + 3 * q
    iw, it_, iu, iv1, iv2 = 0, p, 2 * p, 2 * p + q, 2 * p + 2 * q
    l = 2 * p + q
    m = l + 6 * q
    rows, cols, vals = [], [], []
    b = np.zeros(m)

    def put(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for j in range(p):
        put(j, iw + j, 1.0)
        put(j, it_ + j, -1.0)
        put(p + j, iw + j, -1.0)
        put(p + j, it_ + j, -1.0)
    for i in range(q):
        put(2 * p + i, iv1 + i, 1.0)
        put(2 * p + i, iv2 + i, 1.0)
        b[2 * p + i] = 1.0
    for i in range(q):
        e0 = l + 6 * i
        put(e0, iv1 + i, -1.0)
        b[e0 + 1] = 1.0
        for j in np.nonzero(Asmp[i])[0]:
            put(e0 + 2, iw + j, -Asmp[i, j])
        put(e0 + 2, iu + i, 1.0)
        put(e0 + 3, iv2 + i, -1.0)
        b[e0 + 4] = 1.0
        put(e0 + 5, iu + i, 1.0)
    A = _csr(np.array(rows, np.int64), np.array(cols, np.int64), np.array(vals), m, n)
    c = np.concatenate([np.zeros(p), lam * np.ones(p), np.ones(q), np.zeros(2 * q)])
    return dict(A=A, b=b, c=c, f=0, l=l, q=[], s=[], ep=2 * q, ed=0,
                meta=dict(p=p, q=q, lam=lam, samples=Asmp, w0=w0))


def lasso_paper(seed=0, n=631, kappa=10.0, mu_frac=0.1, frac_nz=0.1, noise=0.01):
    """The LASSO family of Sec. 5.3: F of m = ceil(n/5) rows and n columns with
    condition number kappa, in the epigraph form of `lasso`.  Readings (the
    paper does not say how kappa is imposed or what scale mu has): F = U
    diag(sigma) V^T with U, V orthonormal (QR of Gaussians) and sigma
    log-spaced from 1 down to 1/kappa; mu = mu_frac ||F^T g||_inf (mu_frac in
    {0.01, 0.1, 1}; at 1 the minimiser is 0); x planted with frac_nz N(0,1)
    nonzeros, g = F x + noise N(0,1)."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(n / 5))
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, m)))
    sig = kappa ** (-np.arange(m) / max(m - 1, 1))
    F = (U * sig) @ V.T
    xt = np.zeros(n)
    idx = rng.choice(n, size=max(1, int(round(frac_nz * n))), replace=False)
    xt[idx] = rng.standard_normal(idx.size)
    g = F @ xt + noise * rng.standard_normal(m)
    P = lasso(F=sp.csr_matrix(F), g=g, mu_frac=mu_frac)
    P["meta"].update(kappa=kappa, sigma=sig, xplant=xt)
    return P


def pca_sdp(seed=0, d=50, lam=2.0, k_nz=None, spike=5.0):
    """The sparse PCA SDP of Sec. 5.2, maximise trace(S Z) - lam ||Z||_1 subject
    to trace(Z) = 1, Z PSD, as a cone program in z = svec(Z) and t >= |z|:
        minimise -<svec(S), z> + lam (sum_diag t + sqrt2 sum_offdiag t)
    (svec scales off-diagonal entries by sqrt2, so sum_{i != j} |Z_ij| is
    sqrt2 times the off-diagonal |z|).  Rows: one zero-cone row trace(Z) = 1,
    orthant rows t - z >= 0 and t + z >= 0, one PSD block s = z of order d.
    S (a reading; the paper gives no recipe): a sample covariance B B^T / (2d)
    of a d x 2d Gaussian B plus spike * v v^T with v a unit vector of k_nz
    (default d/10) nonzeros."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((d, 2 * d))
    k_nz = max(1, d // 10) if k_nz is None else k_nz
    v = np.zeros(d)
    idx = rng.choice(d, size=k_nz, replace=False)
    v[idx] = rng.standard_normal(k_nz)
    v /= np.linalg.norm(v)
    S = B @ B.T / (2 * d) + spike * np.outer(v, v)
    k = d * (d + 1) // 2
    sv = _svec(S)
    diag = np.zeros(k, bool)
    o = 0
    for j in range(d):
        diag[o] = True
        o += d - j
    n = 2 * k
    rows, cols, vals = [], [], []
    dz = np.nonzero(diag)[0]
    rows += [0] * len(dz); cols += list(dz); vals += [1.0] * len(dz)
    e = np.arange(k)
    rows += list(1 + e); cols += list(e); vals += [1.0] * k              # t - z >= 0
    rows += list(1 + e); cols += list(k + e); vals += [-1.0] * k
    rows += list(1 + k + e); cols += list(e); vals += [-1.0] * k         # t + z >= 0
    rows += list(1 + k + e); cols += list(k + e); vals += [-1.0] * k
    rows += list(1 + 2 * k + e); cols += list(e); vals += [-1.0] * k     # s = z in the PSD cone
    m = 1 + 3 * k
    A = _csr(np.array(rows), np.array(cols), np.array(vals), m, n)
    b = np.zeros(m)
    b[0] = 1.0
    c = np.concatenate([-sv, lam * np.where(diag, 1.0, math.sqrt(2.0))])
    return dict(A=A, b=b, c=c, f=1, l=2 * k, q=[], s=[d], meta=dict(S=S, lam=lam, d=d, v=v))


def sgm(times, sigma=10.0):
    """Shifted geometric mean of Sec. 5.1 with shift sigma (seconds): failed
    problems (inf or nan) count as 100 times the largest finite time; the
    printed formula lacks the 1/|P| of a mean, read here as
    exp(mean(ln(max(1, sigma + t)))) - sigma."""
    t = np.asarray(times, float)
    ok = np.isfinite(t)
    if not ok.any():
        return float("inf")
    t = np.where(ok, t, 100.0 * t[ok].max())
    return float(np.exp(np.mean(np.log(np.maximum(1.0, sigma + t)))) - sigma)
