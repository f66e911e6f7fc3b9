"""GPU solves of the paper's synthetic families (Sec. 5.2-5.4) at small sizes
against the oracle: status, recomputed KKT residuals, objective and cone
membership, on both execution teams."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import binding as B
from paper_1903_06477_gb300 import workloads as W
from tests.helpers import check_in_cone

pytestmark = pytest.mark.gpu

FAMILIES = {
    "lasso_kappa10": lambda: W.lasso_paper(seed=11, n=120, kappa=10.0, mu_frac=0.1),
    "lasso_kappa1e5": lambda: W.lasso_paper(seed=12, n=120, kappa=1e5, mu_frac=0.01),
    "pca_d20": lambda: W.pca_sdp(seed=13, d=20, lam=2.0),
    "pca_d50": lambda: W.pca_sdp(seed=14, d=50, lam=0.1),
    "logreg": lambda: W.logreg(seed=15, p=30, q=50, lam=10.0),
}


@pytest.mark.parametrize("team", [B.TEAM_BLOCK, B.TEAM_GRID])
@pytest.mark.parametrize("name", list(FAMILIES))
def test_family_solve_matches_oracle(name, team):
    prob = FAMILIES[name]()
    eps = 1e-6
    kw = dict(direction=B.DIR_AA, mem=10, eps=eps, max_iters=50000, cg_rtol=1e-12)
    x, y, s, info = B.Work(prob, team=team, **kw).solve()
    ref = O.Oracle(prob, **kw).solve()
    assert info["status"] == B.SOLVED == ref["info"].status, (info, ref["info"])
    A, b, c = prob["A"], prob["b"], prob["c"]
    pr = np.linalg.norm(A @ x + s - b) / (1 + np.linalg.norm(b))
    dr = np.linalg.norm(A.T @ y + c) / (1 + np.linalg.norm(c))
    assert max(pr, dr) <= 1.01 * eps
    assert abs(info["pobj"] - ref["info"].pobj) <= 10 * eps * (1 + abs(ref["info"].pobj))
    check_in_cone(prob, s, dual=False, tol=1e-6 * (1 + np.abs(s).max()))
    check_in_cone(prob, y, dual=True, tol=1e-6 * (1 + np.abs(y).max()))
