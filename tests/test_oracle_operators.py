"""Pins for (I+Q)^{-1}, T and R (Sec. 3.1 and 4.1 of the paper).

(I+Q)^{-1} is checked against a dense numpy solve of the matrix Q written out
from its definition; T against firm nonexpansiveness, positive homogeneity
and the planted fixed point u* = (x*, y* + s*, 1), which ties together the
signs of Q, the cone conventions and the projection.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import workloads as W
from tests.helpers import dense_Q


def _small_problems():
    return [
        ("lasso", W.lasso(seed=1, p=12, nvar=20, k_nz=4, density=0.3)),
        ("planted", W.planted(seed=2, n=40, l=30, soc=[3, 5, 1], psd=[2, 3], f=3, nnz=400)),
        ("portfolio", W.portfolio(seed=3, k=25)),
    ]


@pytest.mark.parametrize("name,prob", _small_problems())
def test_Q_skew_and_linsys_vs_dense(name, prob):
    orc = O.Oracle(prob, cg_rtol=1e-14, cg_max=5000)
    Q = dense_Q(prob["A"], prob["b"], prob["c"])
    N = Q.shape[0]
    rng = np.random.default_rng(0)
    u = rng.standard_normal(N)
    assert abs(u @ Q @ u) <= 1e-12 * (u @ u) * np.abs(Q).max()
    for slot in (0, 1, 0):
        r = rng.standard_normal(N) * 5
        ref = np.linalg.solve(np.eye(N) + Q, r)
        out = orc.linsys(r, slot=slot)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("name,prob", _small_problems())
def test_T_against_dense_definition(name, prob):
    """Tu = u + Pi_C(2 u~ - u) - u~ with u~ from the dense solve."""
    orc = O.Oracle(prob, cg_rtol=1e-14, cg_max=5000)
    Q = dense_Q(prob["A"], prob["b"], prob["c"])
    N = Q.shape[0]
    rng = np.random.default_rng(1)
    for _ in range(3):
        u = rng.standard_normal(N)
        ut = np.linalg.solve(np.eye(N) + Q, u)
        Tu_ref = u + orc.proj_C(2 * ut - u) - ut
        Tu, Ru = orc.apply_T(u)
        np.testing.assert_allclose(Tu, Tu_ref, atol=1e-9 * (1 + np.abs(u).max()))
        np.testing.assert_allclose(Ru, u - Tu, atol=1e-14 * (1 + np.abs(u).max()))


@pytest.mark.parametrize("name,prob", _small_problems())
def test_T_firmly_nonexpansive_and_homogeneous(name, prob):
    orc = O.Oracle(prob, cg_rtol=1e-14, cg_max=5000)
    N = orc.N
    rng = np.random.default_rng(2)
    for _ in range(10):
        u, v = rng.standard_normal(N) * 3, rng.standard_normal(N) * 3
        Tu, _ = orc.apply_T(u)
        Tv, _ = orc.apply_T(v)
        lhs = np.sum((Tu - Tv) ** 2)
        rhs = (Tu - Tv) @ (u - v)
        assert lhs <= rhs + 1e-9 * (1 + rhs)
        a = rng.uniform(0.1, 10)
        Tau, _ = orc.apply_T(a * u)
        np.testing.assert_allclose(Tau, a * Tu, atol=1e-9 * a * (1 + np.abs(Tu).max()))


def test_planted_fixed_point():
    """u* = (x*, y* + s*, 1) is a fixed point of T for a planted optimum."""
    prob = W.planted(seed=4, n=60, l=50, soc=[4, 6, 2], psd=[3, 2], f=2, nnz=900)
    orc = O.Oracle(prob, cg_rtol=1e-15, cg_max=10000)
    ustar = np.concatenate([prob["xstar"], prob["ystar"] + prob["sstar"], [1.0]])
    _, Ru = orc.apply_T(ustar)
    assert np.linalg.norm(Ru) <= 1e-9 * np.linalg.norm(ustar)
    # and a perturbed point is not
    _, Ru2 = orc.apply_T(ustar + 0.1)
    assert np.linalg.norm(Ru2) > 1e-3


def test_termination_on_planted_point():
    """At u* the termination test sees pr = dr = gap = 0 and sigma_ in K, <y_, s_> = 0."""
    prob = W.planted(seed=7, n=50, l=40, soc=[5, 5], f=1, nnz=700)
    orc = O.Oracle(prob, cg_rtol=1e-15, cg_max=10000)
    n = 50
    ustar = np.concatenate([prob["xstar"], prob["ystar"] + prob["sstar"], [1.0]])
    ut = orc.linsys(ustar)
    ub = orc.proj_C(2 * ut - ustar)
    st, info = orc.termination(ustar, ut, ub, 1e-8)
    assert st == O.SOLVED
    assert max(info.pr, info.dr, info.gap) <= 1e-9
    np.testing.assert_allclose(info.pobj, prob["c"] @ prob["xstar"], rtol=1e-9)
    # sigma_ = psi_ - 2 psi~ + psi equals Pi_K(psi - 2 psi~) and is orthogonal to psi_
    sig = ub[n:-1] - 2 * ut[n:-1] + ustar[n:-1]
    np.testing.assert_allclose(sig, orc.proj_primal_cone(ustar[n:-1] - 2 * ut[n:-1]), atol=1e-9)
    assert abs(sig @ ub[n:-1]) <= 1e-9 * (1 + np.abs(sig).max() * np.abs(ub).max())
