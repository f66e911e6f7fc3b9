"""Pins for the quasi-Newton directions (Sec. 4.4 of the paper).

Restarted Broyden (Algorithm 2) is checked against the full-memory recursion
it implements: H_{k+1} = H_k + (z - H_k xi~)(z^T H_k) / <z, H_k xi~> with
Powell's theta safeguard, carried out with dense N x N matrices.  Anderson's
acceleration is checked against numpy.linalg.lstsq and the orthogonality of
the least-squares residual.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _theta(gamma, tb):
    if abs(gamma) >= tb:
        return 1.0
    sg = 1.0 if gamma >= 0 else -1.0
    return (1 - sg * tb) / (1 - gamma)


@pytest.mark.parametrize("mem", [3, 5, 10])
def test_rb_matches_dense_sherman_morrison(mem):
    N, tb = 30, 0.1
    rng = np.random.default_rng(mem)
    D = O.Direction(O.DIR_RB, N, mem, thetabar=tb)
    H = np.eye(N)
    theta_small = 0
    for it in range(2 * mem + 3):
        Ru = rng.standard_normal(N)
        if it == 0:
            d = D(Ru)
            np.testing.assert_allclose(d, -Ru)
            continue
        z = rng.standard_normal(N)
        # xi close to J z for a fixed nonsymmetric J, sometimes with small gamma
        J = np.eye(N) + 0.3 * np.random.default_rng(99).standard_normal((N, N)) / np.sqrt(N)
        if it % 3 == 0:
            # H xi = 0.05 z + (something orthogonal to z): gamma = 0.05 < thetabar
            o = rng.standard_normal(N)
            o -= (o @ z) / (z @ z) * z
            xi = np.linalg.solve(H, 0.05 * z + o)
        else:
            xi = J @ z
        count_before = D.count
        d = D(Ru, z, xi)
        # dense: B-update with Powell's theta, H via Sherman-Morrison (full memory since last restart)
        gamma = (H @ xi) @ z / (z @ z)
        th = _theta(gamma, tb)
        theta_small += th != 1.0
        Hxi_t = (1 - th) * z + th * (H @ xi)  # H xi~ with xi~ = (1-th) B z + th xi, H B = I
        Hn = H + np.outer(z - Hxi_t, z @ H) / (z @ Hxi_t)
        np.testing.assert_allclose(d, -Hn @ Ru, rtol=0, atol=1e-9 * (1 + np.abs(d).max()))
        if count_before == mem:
            H = np.eye(N)  # restart: buffers emptied, current pair not stored
            assert D.count == 0
        else:
            H = Hn
            assert D.count == count_before + 1
    assert theta_small > 0  # the safeguard branch was exercised


def test_rb_mem0_uses_only_current_pair():
    N = 12
    rng = np.random.default_rng(5)
    D = O.Direction(O.DIR_RB, N, 0)
    D(rng.standard_normal(N))
    for _ in range(3):
        Ru, z, xi = rng.standard_normal((3, N))
        d = D(Ru, z, xi)
        gamma = xi @ z / (z @ z)
        th = _theta(gamma, 0.1)
        Hxi_t = (1 - th) * z + th * xi
        H = np.eye(N) + np.outer(z - Hxi_t, z) / (z @ Hxi_t)
        np.testing.assert_allclose(d, -H @ Ru, atol=1e-10)
        assert D.count == 0


@pytest.mark.parametrize("kind", [O.DIR_AA, O.DIR_AA_QR])
@pytest.mark.parametrize("mem", [1, 3, 5, 10])
def test_aa_matches_lstsq(mem, kind):
    # both least-squares solvers of the AA direction (regularised normal equations, and
    # the QR factorisation updated as pairs enter and leave the window) against lstsq
    N = 40
    rng = np.random.default_rng(20 + mem)
    D = O.Direction(kind, N, mem, aa_reg=1e-14)
    Zs, Xs = [], []
    D(rng.standard_normal(N))
    for it in range(2 * mem + 2):
        Ru = rng.standard_normal(N)
        z, xi = rng.standard_normal(N), rng.standard_normal(N)
        d = D(Ru, z, xi)
        Zs.append(z); Xs.append(xi)
        Zs, Xs = Zs[-mem:], Xs[-mem:]
        Z, X = np.array(Zs).T, np.array(Xs).T
        t, *_ = np.linalg.lstsq(X, Ru, rcond=None)
        ref = -Ru - (Z - X) @ t
        np.testing.assert_allclose(d, ref, atol=1e-8 * (1 + np.abs(ref).max()))
        # least-squares optimality: Xi^T (Xi t - Ru) = 0
        assert np.abs(X.T @ (X @ t - Ru)).max() <= 1e-8 * (1 + np.abs(Ru).max())
        assert D.count == min(it + 1, mem)


def test_aa_linear_residual_gives_anderson_step():
    """For an affine R(u) = J u - r0 with a full history, AA's d makes
    R(u + d) = (I - J)(Ru - Xi t): the type-II Anderson identity."""
    N, mem = 25, 6
    rng = np.random.default_rng(7)
    J = np.eye(N) * 0.5 + 0.1 * rng.standard_normal((N, N))
    r0 = rng.standard_normal(N)
    R = lambda u: J @ u - r0
    D = O.Direction(O.DIR_AA, N, mem, aa_reg=1e-14)
    u = rng.standard_normal(N)
    D(R(u))
    Zs, Xs = [], []
    for _ in range(mem):
        w = u + 0.1 * rng.standard_normal(N)
        z, xi = w - u, R(w) - R(u)
        Zs.append(z); Xs.append(xi)
        u = w
        d = D(R(u), z, xi)
    X = np.array(Xs).T
    t, *_ = np.linalg.lstsq(X, R(u), rcond=None)
    lhs = R(u + d)
    rhs = (np.eye(N) - J) @ (R(u) - X @ t)
    np.testing.assert_allclose(lhs, rhs, atol=1e-8)


def test_aa_mem0_is_minus_residual():
    N = 10
    D = O.Direction(O.DIR_AA, N, 0)
    rng = np.random.default_rng(0)
    D(rng.standard_normal(N))
    Ru = rng.standard_normal(N)
    np.testing.assert_allclose(D(Ru, rng.standard_normal(N), rng.standard_normal(N)), -Ru)


def test_aa_qr_skips_rank_deficient_pair():
    # a pair whose xi lies in the span of the stored ones is not stored by the QR variant
    N = 20
    rng = np.random.default_rng(8)
    D = O.Direction(O.DIR_AA_QR, N, 4)
    D(rng.standard_normal(N))
    x1, x2 = rng.standard_normal(N), rng.standard_normal(N)
    D(rng.standard_normal(N), rng.standard_normal(N), x1)
    D(rng.standard_normal(N), rng.standard_normal(N), x2)
    assert D.count == 2
    D(rng.standard_normal(N), rng.standard_normal(N), 0.3 * x1 - 2.0 * x2)
    assert D.count == 2
