"""Parity at the full benchmark sizes, in the launch configurations bench.py
times.

Whole solves at these sizes take the oracle minutes to hours, so the checks
are (1) one application of the operator T (Eq. drs: the linear-system step
by CG plus the cone projection) on the full instance against the oracle,
element by element, and (2) the benchmark's own solve judged by what holds
at any size: the KKT residuals of Sec. 4.3 recomputed here in FP64 from the
returned (x, y, s), cone membership, and the planted optimum c^T x*.

Tolerance of (1): both sides run CG to ||res|| <= 1e-13 ||rhs|| on
I + A^T A, whose condition number is 1 + sigma_max(A)^2 (a few hundred for
these random matrices), so the solutions agree to about 1e-10 relative; the
test allows 1e-8 of the largest entry.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import binding as B
from paper_1903_06477_gb300 import workloads as W
from tests.helpers import check_in_cone

pytestmark = pytest.mark.gpu

TOL_T = 1e-8


def _kkt(prob, x, y, s):
    A, b, c = prob["A"], prob["b"], prob["c"]
    pr = np.linalg.norm(A @ x + s - b) / (1 + np.linalg.norm(b))
    dr = np.linalg.norm(A.T @ y + c) / (1 + np.linalg.norm(c))
    cx, by = c @ x, b @ y
    gap = abs(cx + by) / (1 + abs(cx) + abs(by))
    return pr, dr, gap


def _T_parity(prob, **kw):
    work = B.Work(prob, cg_rtol=1e-13, cg_max=5000, **kw)
    orc = O.Oracle(prob, cg_rtol=1e-13, cg_max=5000)
    rng = np.random.default_rng(17)
    u = rng.standard_normal(work.N)
    u[-1] = 1.0
    Tu, Ru = work.apply_T(u)
    Tr, Rr = orc.apply_T(u)
    scale = 1 + np.abs(Tr).max()
    np.testing.assert_allclose(Tu, Tr, rtol=0, atol=TOL_T * scale)
    np.testing.assert_allclose(Ru, Rr, rtol=0, atol=TOL_T * scale)
    work.close()
    orc.close()


@pytest.fixture(scope="module")
def c2():
    return W.c2_planted(seed=0)


def test_c2_full_operator_T_matches_oracle(c2):
    """n = 100k, m = 200k, 1e7 nonzeros; grid team, column-blocked products."""
    _T_parity(c2)


def test_c2_full_bench_solve(c2):
    """The benchmark's configuration: AA(10), eps 1e-6, FP32 phase with FP64
    refinement, adaptive CG tolerance."""
    eps = 1e-6
    kw = dict(direction=0, mem=10, eps=eps, max_iters=20000, cg_rtol=1e-10, cg_adapt=1e-2, mixed_switch=3e-5)
    work = B.Work(c2, precision=B.MIXED, **kw)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    assert max(_kkt(c2, x, y, s)) <= eps * 1.01
    check_in_cone(c2, s, dual=False, tol=1e-7 * (1 + np.abs(s).max()))
    check_in_cone(c2, y, dual=True, tol=1e-7 * (1 + np.abs(y).max()))
    pstar = c2["c"] @ c2["xstar"]
    assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))
    assert info["iters_fp32"] > 0


@pytest.fixture(scope="module")
def c3():
    return W.c3_planted_sdp(seed=0)


def test_c3_full_operator_T_matches_oracle(c3):
    """512 PSD blocks of order 64 plus 50k orthant rows, 1e6 nonzeros: the
    batched Jacobi eigensolves of the projection against the oracle's."""
    _T_parity(c3)


def test_c3_full_bench_solve(c3):
    eps = 1e-4
    kw = dict(direction=0, mem=10, eps=eps, max_iters=20000, cg_rtol=1e-10, cg_adapt=1e-2, mixed_switch=1e-4)
    work = B.Work(c3, precision=B.MIXED, **kw)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    assert max(_kkt(c3, x, y, s)) <= eps * 1.01
    check_in_cone(c3, s, dual=False, tol=1e-6 * (1 + np.abs(s).max()))
    check_in_cone(c3, y, dual=True, tol=1e-6 * (1 + np.abs(y).max()))
    pstar = c3["c"] @ c3["xstar"]
    assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))
    assert 0 < info["psd_resid_fp32"] < 1e-4


def test_c4_full_batch():
    """4096 portfolio SOCPs (k ~ U{20..400}) in one persistent launch per
    phase, FP32 bulk with FP64 refinement, linear systems by the dense
    Cholesky factor (the benchmark's form), eps 1e-5: every instance solved
    with its KKT residuals at eps; a sample against the oracle's solve."""
    probs = W.c4_portfolios(4096)
    eps = 1e-5
    kw = dict(direction=0, mem=10, eps=eps, max_iters=20000, cg_rtol=1e-10, cg_adapt=1e-2, mixed_switch=1e-5,
              linsys_direct=1)
    batch = B.Batch(probs, precision=B.MIXED, **kw)
    xs, ys, ss, infos = batch.solve()
    for p, x, y, s, info in zip(probs, xs, ys, ss, infos):
        assert info["status"] == B.SOLVED, info
        assert max(_kkt(p, x, y, s)) <= eps * 1.01
    okw = dict(direction=O.DIR_AA, mem=10, eps=eps, max_iters=20000, cg_rtol=1e-10)
    for i in range(0, 4096, 683):
        ref = O.Oracle(probs[i], **okw).solve()
        assert ref["info"].status == O.SOLVED
        p_ref = ref["info"].pobj
        assert abs(infos[i]["pobj"] - p_ref) <= 10 * eps * (1 + abs(p_ref)), (i, infos[i]["pobj"], p_ref)


def test_c5_full_family_operator_and_batch():
    """Parametric LASSO family, F 2000 x 5000 at 1% (n = 10001, m = 12002):
    T against the oracle on one member, then a shared-matrix batch of 256
    members in the benchmark's configuration, each solved to eps."""
    F = W.lasso_family_matrix(seed=0)
    prob0 = W.lasso(F=F, g=W.lasso_family_rhs(F, seed=1))
    _T_parity(prob0)
    eps = 1e-5
    kw = dict(direction=B.DIR_RB, mem=10, c0=0.1, precision=B.FP64, eps=eps, max_iters=20000, cg_adapt=1e-2,
              warm_fallback=50)
    gs = [W.lasso_family_rhs(F, seed=200_000 + i) for i in range(256)]
    bcs = [W.lasso_family_bc(F, g) for g in gs]
    batch = B.Batch(shared=(prob0, [b for b, _ in bcs], [c for _, c in bcs]), **kw)
    xs, ys, ss, infos = batch.solve()
    for (b, c), x, y, s, info in zip(bcs, xs, ys, ss, infos):
        assert info["status"] == B.SOLVED, info
        p = dict(prob0, b=b, c=c)
        assert max(_kkt(p, x, y, s)) <= eps * 1.01
