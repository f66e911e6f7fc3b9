"""The paper's synthetic families (Sec. 5.2-5.4) and the shifted geometric
mean of Sec. 5.1: generators and the oracle's solves pinned by closed forms
and an independent solver."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import workloads as W
from tests.helpers import check_in_cone, fista_lasso, svec_mat


def test_sgm_hand_values():
    # equal times t give t; a failure counts as 100 x the largest finite time; the shift sigma
    assert W.sgm([2.0, 2.0, 2.0]) == pytest.approx(2.0)
    assert W.sgm([1.0, np.inf]) == pytest.approx(np.sqrt(11.0 * 110.0) - 10.0)
    assert W.sgm([0.0, 0.0], sigma=0.0) == pytest.approx(1.0)  # max(1, .) floors every term at 1
    assert W.sgm([3.0, 27.0], sigma=0.0) == pytest.approx(9.0)


@pytest.mark.parametrize("kappa", [10.0, 4600.0])
def test_lasso_family_condition_and_fista(kappa):
    P = W.lasso_paper(seed=2, n=80, kappa=kappa, mu_frac=0.1)
    F = P["meta"]["F"].toarray()
    assert F.shape == (16, 80)
    assert np.linalg.cond(F) == pytest.approx(kappa, rel=1e-9)
    out = O.Oracle(P, eps=1e-9, max_iters=100000).solve()
    assert out["info"].status == O.SOLVED
    x = out["x"][:80]
    xf = fista_lasso(F, P["meta"]["g"], P["meta"]["mu"], iters=60000)
    obj = lambda v: 0.5 * np.sum((F @ v - P["meta"]["g"]) ** 2) + P["meta"]["mu"] * np.abs(v).sum()
    assert abs(obj(x) - obj(xf)) <= 1e-7 * (1 + abs(obj(xf)))


def test_lasso_family_mu_one_gives_zero():
    # mu = ||F^T g||_inf: 0 satisfies the subgradient condition, so the minimiser is 0
    P = W.lasso_paper(seed=3, n=60, kappa=10.0, mu_frac=1.0)
    out = O.Oracle(P, eps=1e-9, max_iters=100000).solve()
    assert out["info"].status == O.SOLVED
    assert np.abs(out["x"][:60]).max() <= 1e-6


def test_pca_lambda_zero_is_top_eigenvalue():
    # without the l1 term the optimum of max trace(SZ), trace Z = 1, Z PSD is lambda_max(S)
    P = W.pca_sdp(seed=4, d=9, lam=0.0)
    out = O.Oracle(P, eps=1e-9, max_iters=50000).solve()
    assert out["info"].status == O.SOLVED
    assert out["info"].pobj == pytest.approx(-np.linalg.eigvalsh(P["meta"]["S"]).max(), abs=1e-7)


def test_pca_feasible_and_bounded_by_rank_one_candidates():
    P = W.pca_sdp(seed=5, d=10, lam=2.0)
    S, lam, d = P["meta"]["S"], 2.0, 10
    out = O.Oracle(P, eps=1e-8, max_iters=50000).solve()
    assert out["info"].status == O.SOLVED
    k = d * (d + 1) // 2
    Z = svec_mat(out["x"][:k], d)
    assert abs(np.trace(Z) - 1) <= 1e-6 and np.linalg.eigvalsh(Z).min() >= -1e-6
    check_in_cone(P, out["s"], dual=False, tol=1e-6)
    opt = np.trace(S @ Z) - lam * np.abs(Z).sum()
    assert opt == pytest.approx(-out["info"].pobj, abs=1e-5)
    # every feasible Z = v v^T (unit v) is no better than the optimum
    rng = np.random.default_rng(0)
    for v in list(np.linalg.eigh(S)[1].T) + list(rng.standard_normal((50, d))):
        v = v / np.linalg.norm(v)
        Zc = np.outer(v, v)
        assert np.trace(S @ Zc) - lam * np.abs(Zc).sum() <= opt + 1e-6
