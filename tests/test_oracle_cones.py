"""Pins for the oracle's cone projections (Sec. 2 of the paper).

Each projection is pinned by something other than itself: hand-worked cases
of the closed form (tests/golden), the Moreau decomposition, which determines
the projection uniquely (v = a - b, a in K, b in K*, <a,b> = 0 => a = Pi_K v),
idempotence, the variational inequality, and numpy.linalg.eigh for PSD.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import workloads as W
from tests.helpers import check_in_cone, in_soc, read_cases, svec_mat


@pytest.mark.parametrize("case", read_cases("soc_projection_cases.txt"))
def test_soc_golden(case):
    zin, zout = np.array(case[0]), np.array(case[1])
    np.testing.assert_allclose(O.proj_soc(zin), zout, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dim", [1, 2, 3, 5, 50, 62, 400])
def test_soc_moreau_and_vi(dim):
    rng = np.random.default_rng(dim)
    for trial in range(40):
        v = rng.standard_normal(dim) * rng.uniform(0.1, 10)
        if trial % 4 == 1:
            v[-1] = np.linalg.norm(v[:-1]) * rng.uniform(-1.5, 1.5)
        a = O.proj_soc(v)
        bneg = O.proj_soc(-v)
        # Moreau (SOC is self-dual): v = Pi_K(v) - Pi_K(-v), <Pi_K v, Pi_K(-v)> = 0
        np.testing.assert_allclose(a - bneg, v, atol=1e-12 * (1 + np.abs(v).max()))
        assert abs(a @ bneg) <= 1e-11 * (1 + v @ v)
        assert in_soc(a) and in_soc(bneg)
        # idempotent
        np.testing.assert_allclose(O.proj_soc(a), a, atol=1e-13 * (1 + np.abs(a).max()))
        # variational inequality against random cone points
        for _ in range(5):
            x = rng.standard_normal(dim - 1) if dim > 1 else np.zeros(0)
            k = np.concatenate([x, [np.linalg.norm(x) + rng.uniform(0, 2)]])
            assert (v - a) @ (k - a) <= 1e-10 * (1 + v @ v)


@pytest.mark.parametrize("case", read_cases("psd_projection_cases.txt"))
def test_psd_golden(case):
    d = int(case[0][0])
    vin, vout = np.array(case[1]), np.array(case[2])
    np.testing.assert_allclose(O.proj_psd(vin, d), vout, rtol=0, atol=1e-13)


def test_svec_mat_inner_product():
    rng = np.random.default_rng(3)
    for d in (1, 2, 3, 7, 16):
        k = d * (d + 1) // 2
        x, y = rng.standard_normal(k), rng.standard_normal(k)
        X, Y = O.svec_to_mat(x, d), O.svec_to_mat(y, d)
        np.testing.assert_allclose(X, svec_mat(x, d), atol=1e-15)
        # <x,y> = tr(mat x mat y): the reason for the sqrt(2) scaling
        assert abs(x @ y - np.trace(X @ Y)) <= 1e-12 * (1 + abs(x @ y))
        np.testing.assert_allclose(O.mat_to_svec(X), x, atol=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 20, 64])
def test_jacobi_vs_eigh(d):
    rng = np.random.default_rng(d)
    G = rng.standard_normal((d, d))
    X = 0.5 * (G + G.T)
    lam, V = O.jacobi_eig(X)
    ref = np.linalg.eigvalsh(X)
    np.testing.assert_allclose(np.sort(lam), ref, atol=1e-12 * (1 + np.abs(ref).max()))
    # eigen-residual and orthogonality
    assert np.linalg.norm(X @ V - V * lam) <= 1e-12 * np.linalg.norm(X) * d
    np.testing.assert_allclose(V.T @ V, np.eye(d), atol=1e-12 * d)


def test_jacobi_2x2_closed_form():
    # eigenvalues of [[a,b],[b,c]] are (a+c)/2 +- sqrt(((a-c)/2)^2 + b^2)
    rng = np.random.default_rng(11)
    for _ in range(50):
        a, bb, c = rng.standard_normal(3)
        lam, _ = O.jacobi_eig(np.array([[a, bb], [bb, c]]))
        r = np.hypot((a - c) / 2, bb)
        np.testing.assert_allclose(np.sort(lam), [(a + c) / 2 - r, (a + c) / 2 + r], atol=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 12])
def test_psd_projection_vs_eigh(d):
    rng = np.random.default_rng(100 + d)
    k = d * (d + 1) // 2
    for _ in range(10):
        v = rng.standard_normal(k)
        X = svec_mat(v, d)
        w, U = np.linalg.eigh(X)
        Xp = (U * np.maximum(w, 0)) @ U.T
        ref = np.array([Xp[i, j] * (1 if i == j else np.sqrt(2)) for j in range(d) for i in range(j, d)])
        out = O.proj_psd(v, d)
        np.testing.assert_allclose(out, ref, atol=1e-12 * (1 + np.abs(v).max()))
        # Moreau: v = Pi(v) - Pi(-v), orthogonal
        neg = O.proj_psd(-v, d)
        np.testing.assert_allclose(out - neg, v, atol=1e-12 * (1 + np.abs(v).max()))
        assert abs(out @ neg) <= 1e-11 * (1 + v @ v)


def test_mixed_cone_moreau_and_zero_cone():
    """Pi_K and Pi_K* over [f | l | q | s]: zero-cone rows are 0 under K and free under K*."""
    prob = W.planted(seed=5, n=30, l=7, soc=[1, 2, 5], psd=[1, 3], f=4, nnz=200)
    orc = O.Oracle(prob)
    rng = np.random.default_rng(0)
    m = prob["A"].shape[0]
    for _ in range(20):
        v = rng.standard_normal(m) * 3
        pk = orc.proj_primal_cone(v)
        pd = orc.proj_dual_cone(-v)
        # Moreau for K: v = Pi_K(v) - Pi_{K*}(-v), <Pi_K(v), Pi_{K*}(-v)> = 0
        np.testing.assert_allclose(pk - pd, v, atol=1e-12 * (1 + np.abs(v).max()))
        assert abs(pk @ pd) <= 1e-11 * (1 + v @ v)
        check_in_cone(prob, pk, dual=False, tol=1e-12)
        check_in_cone(prob, pd, dual=True, tol=1e-12)
        assert np.all(pk[:4] == 0)
        np.testing.assert_array_equal(orc.proj_dual_cone(v)[:4], v[:4])


def test_proj_C_structure():
    """Pi_C with C = R^n x K* x R_+: chi untouched, tau clipped at 0."""
    prob = W.planted(seed=6, n=20, l=10, soc=[4], f=2, nnz=100)
    orc = O.Oracle(prob)
    n, m = 20, prob["A"].shape[0]
    rng = np.random.default_rng(1)
    v = rng.standard_normal(n + m + 1)
    v[-1] = -0.5
    out = orc.proj_C(v)
    np.testing.assert_array_equal(out[:n], v[:n])
    assert out[-1] == 0.0
    np.testing.assert_allclose(out[n:n + m], orc.proj_dual_cone(v[n:n + m]))


# --- exponential cone (Sec. 2, cone (v)): K^e = cl{x1 >= x2 exp(x3/x2), x2 > 0} ---------------------------
_RHO = np.concatenate([-np.logspace(3, -3, 400), [0.0], np.linspace(-60, 60, 24001), np.logspace(-3, 3, 400)])


def _gens_K():
    # extreme rays of K^e, normalised: x2 = 1, x3 = rho, x1 = e^rho, and the face rays (1,0,0), (0,0,-1)
    rho = _RHO[np.abs(_RHO) < 350]
    G = np.stack([np.exp(rho), np.ones_like(rho), rho], 1)
    G = np.vstack([G, [[1.0, 0, 0], [0, 0, -1.0]]])
    return G / np.linalg.norm(G, axis=1, keepdims=True)


def _gens_Kdual():
    # extreme rays of (K^e)*: y3 = -1, y2 = -sig, y1 = e^(sig - 1), and the face rays (1,0,0), (0,1,0)
    sig = _RHO[np.abs(_RHO) < 350]
    G = np.stack([np.exp(sig - 1), -sig, -np.ones_like(sig)], 1)
    G = np.vstack([G, [[1.0, 0, 0], [0, 1.0, 0]]])
    return G / np.linalg.norm(G, axis=1, keepdims=True)


_GK, _GKD = _gens_K(), _gens_Kdual()


def _exp_in(x, tol):
    # x in K^e = (K^e)** iff <x, g> >= 0 for every generator g of the dual cone (a distance-like test)
    return (_GKD @ np.asarray(x, float)).min() >= -tol


def _exp_dual_in(y, tol):
    # y in (K^e)* iff <y, g> >= 0 for every generator g of K^e (the definition of a dual cone)
    return (_GK @ np.asarray(y, float)).min() >= -tol


def test_exp_membership_and_closed_forms():
    assert O.in_exp([np.e, 1.0, 1.0]) and O.in_exp([0.0, 0.0, -5.0]) and not O.in_exp([1.0, 1.0, 1.0])
    assert O.in_exp_dual([1.0, 0.0, -np.e]) and O.in_exp_dual([1.0, 2.0, 0.0]) and not O.in_exp_dual([1.0, 0.0, 1.0])
    # a point of the cone is its own projection, a point of the polar cone -(K^e)* goes to 0
    np.testing.assert_array_equal(O.proj_exp([5.0, 1.0, 0.5]), [5.0, 1.0, 0.5])
    np.testing.assert_array_equal(O.proj_exp([-1.0, 0.0, np.e]), [0.0, 0.0, 0.0])
    # x2 <= 0 and x3 <= 0: the face {x2 = 0, x3 <= 0, x1 >= 0}, nearest point (max(x1, 0), 0, x3)
    np.testing.assert_array_equal(O.proj_exp([2.0, -1.0, -3.0]), [2.0, 0.0, -3.0])
    np.testing.assert_array_equal(O.proj_exp([-2.0, -1.0, -3.0]), [0.0, 0.0, -3.0])


def test_exp_projection_of_planted_kkt_points():
    # p on the surface x1 = x2 e^{x3/x2} (x2 = c, x3 = c rho) plus lam times the outward normal
    # n = (-1, e^rho (1 - rho), e^rho) of {x2 e^{x3/x2} - x1 <= 0}: Pi(p + lam n) = p
    rng = np.random.default_rng(3)
    for _ in range(400):
        rho = rng.uniform(-8, 8)
        c = np.exp(rng.uniform(-4, 3))
        lam = np.exp(rng.uniform(-4, 3))
        p = c * np.array([np.exp(rho), 1.0, rho])
        n = np.array([-1.0, np.exp(rho) * (1 - rho), np.exp(rho)])
        got = O.proj_exp(p + lam * n)
        np.testing.assert_allclose(got, p, rtol=0, atol=1e-11 * (1 + np.abs(p).max() + lam * np.abs(n).max()))


def test_exp_projection_kkt_and_moreau_on_random_points():
    rng = np.random.default_rng(4)
    for _ in range(3000):
        v = rng.standard_normal(3) * np.exp(rng.uniform(-3, 3))
        p = O.proj_exp(v)
        q = v - p
        sc = 1e-10 * (1 + np.abs(v).max())
        assert _exp_in(p, sc), (v, p)
        assert _exp_dual_in(-q, sc), (v, p, q)  # v - p in the polar cone -(K^e)*
        assert abs(p @ q) <= sc * (1 + np.abs(v).max()), (v, p)
        np.testing.assert_allclose(O.proj_exp(p), p, rtol=0, atol=sc)  # idempotent
        # the dual projection: Pi_{K*}(v) in K*, v - Pi_{K*}(v) in -K, orthogonal
        pd = O.proj_exp_dual(v)
        qd = v - pd
        assert _exp_dual_in(pd, sc) and _exp_in(-qd, sc) and abs(pd @ qd) <= sc * (1 + np.abs(v).max())


def test_exp_projection_is_nearest_boundary_point_brute_force():
    # brute force on a dense sampling of the boundary: rays c (e^rho, 1, rho) and the face
    rng = np.random.default_rng(5)
    rho = np.linspace(-12, 12, 24001)
    A = np.stack([np.exp(rho), np.ones_like(rho), rho], 1)
    An = A / np.linalg.norm(A, axis=1, keepdims=True)
    for _ in range(300):
        v = rng.standard_normal(3) * np.exp(rng.uniform(-2, 2))
        p = O.proj_exp(v)
        d = np.linalg.norm(v - p)
        cs = np.maximum(An @ v, 0)
        dray = np.sqrt(np.maximum(v @ v - cs ** 2, 0)).min()
        face = np.array([max(v[0], 0), 0.0, min(v[2], 0)])
        dbest = min(dray, np.linalg.norm(v - face), np.linalg.norm(v), 0.0 if _exp_in(v, 0) else np.inf)
        assert d <= dbest + 1e-7 * (1 + np.abs(v).max()), (v, p, d, dbest)
        assert d >= dbest - 1e-3 * (1 + np.abs(v).max())  # the sampling is fine enough to come close


def test_exp_planted_mistake_is_caught():
    # planted mistake, on the CPU: using the wrong element order (x3 read as x1) breaks the KKT pin
    rng = np.random.default_rng(6)
    bad = 0
    for _ in range(50):
        v = rng.standard_normal(3)
        p = O.proj_exp(v[::-1])[::-1]
        q = v - p
        if not (_exp_in(p, 1e-9) and _exp_dual_in(-q, 1e-9) and abs(p @ q) <= 1e-9):
            bad += 1
    assert bad > 10
