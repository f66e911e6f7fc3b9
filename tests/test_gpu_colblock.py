"""GPU parity of the column-blocked sparse products (grid team).

The column-blocked layout cuts A and A^T into column blocks whose slice of
the multiplied vector is staged in shared memory; its products must equal
the plain definition (A x)_i = sum_j a_ij x_j.  The bound used is the
rigorous one for any summation order: |fl(A x) - A x| <= gamma_{k+2} (|A||x|)
with k the longest row and gamma_k = k u / (1 - k u), u the unit roundoff of
the bulk precision (the two extra roundings are those of a_ij and x_j to
FP32; in FP64 they are exact).  spmv_path 3 forces the layout on problems
too small for the automatic rule, so several column blocks, rows ranges
with no rows, skewed row lengths and vectors at odd offsets are all covered.
spmv_path 4 does the same for the two-dimensional tiles, whose sums add the
column blocks' partials in a second pass (k + ncb terms: the bound's k is
raised by the number of column blocks, at most 152).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_1903_06477_gb300 import binding as B
from paper_1903_06477_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24


def _gamma(k, u):
    return k * u / (1 - k * u)


def _skewed(seed=5, n=20001, m=30000):
    """Orthant-only problem whose A mixes a few dense rows and columns, many
    short rows, empty rows and empty columns."""
    rng = np.random.default_rng(seed)
    A = W.random_pattern(rng, m, n, 200_000).tolil()
    for i in rng.choice(m, 6, replace=False):
        cols = rng.choice(n, 4000, replace=False)
        A[i, cols] = rng.standard_normal(4000)
    for j in rng.choice(n, 4, replace=False):
        rows = rng.choice(m, 3000, replace=False)
        A[rows, j] = rng.standard_normal((3000, 1))
    A = A.tocsr()
    empty_r = rng.choice(m, 500, replace=False)
    empty_c = rng.choice(n, 300, replace=False)
    A = sp.diags(np.where(np.isin(np.arange(m), empty_r), 0.0, 1.0)) @ A
    A = A @ sp.diags(np.where(np.isin(np.arange(n), empty_c), 0.0, 1.0))
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    b = rng.uniform(0.5, 1.5, m)
    c = rng.standard_normal(n)
    return dict(A=A, b=b, c=c, f=0, l=m, q=[], s=[])


def _problems():
    return {
        # several column blocks in both precisions; n odd puts y at an odd offset
        "multi_block": W.planted(seed=11, n=30001, l=40000, soc=[50] * 200, nnz=600_000),
        "skewed": _skewed(),
        # fewer rows than CTAs: most row ranges are empty
        "tiny": W.planted(seed=12, n=37, l=40, soc=[5, 8], nnz=500),
    }


PROBS = _problems()


def _check_products(work, prob, precision, u, seed, extra=0):
    A = prob["A"].tocsr()
    AT = A.T.tocsr()
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(work.n)
    y = rng.standard_normal(work.m)
    y2 = rng.uniform(-3, 3, work.m)
    kA = int(np.diff(A.indptr).max(initial=0))
    kT = int(np.diff(AT.indptr).max(initial=0))
    absA, absT = abs(A), abs(AT)
    out = work.spmv(x, op=0, precision=precision)
    bound = _gamma(kA + 2 + extra, u) * (absA @ np.abs(x)) + 1e-300
    assert np.all(np.abs(out - A @ x) <= bound)
    out = work.spmv(y, op=1, precision=precision)
    bound = _gamma(kT + 2 + extra, u) * (absT @ np.abs(y)) + 1e-300
    assert np.all(np.abs(out - AT @ y) <= bound)
    o1, o2 = work.spmv(y, op=2, precision=precision, v2=y2)
    assert np.all(np.abs(o1 - AT @ y) <= bound)
    bound2 = _gamma(kT + 2 + extra, u) * (absT @ np.abs(y2)) + 1e-300
    assert np.all(np.abs(o2 - AT @ y2) <= bound2)


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("path", [4, 3, 1, 2])  # tiles, column-blocked, sliced ELL, sliced ELL with a TMA-staged stream
def test_products_match_definition(name, path):
    prob = PROBS[name]
    work = B.Work(prob, team=B.TEAM_GRID, precision=B.MIXED, spmv_path=path)
    extra = 152 if path == 4 else 0  # the partials of at most 152 column blocks
    _check_products(work, prob, B.FP64, U64, seed=1, extra=extra)
    _check_products(work, prob, B.MIXED, U32, seed=2, extra=extra)
    # a second product right after the first (partial-sum buffers alternate)
    _check_products(work, prob, B.MIXED, U32, seed=3, extra=extra)


@pytest.mark.parametrize("path", [4, 3])
@pytest.mark.parametrize("name", ["multi_block", "skewed"])
def test_column_blocked_linsys_and_T_match_oracle(name, path):
    prob = PROBS[name]
    work = B.Work(prob, team=B.TEAM_GRID, spmv_path=path, cg_rtol=1e-14, cg_max=5000)
    orc = O.Oracle(prob, cg_rtol=1e-14, cg_max=5000)
    rng = np.random.default_rng(3)
    r = rng.standard_normal(work.N) * 3
    out = work.linsys(r, slot=0)
    ref = orc.linsys(r, slot=0)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9 * (1 + np.abs(ref).max()))
    u = rng.standard_normal(work.N)
    Tu, Ru = work.apply_T(u)
    Tr, Rr = orc.apply_T(u)
    np.testing.assert_allclose(Tu, Tr, rtol=0, atol=1e-9 * (1 + np.abs(Tr).max()))
    np.testing.assert_allclose(Ru, Rr, rtol=0, atol=1e-9 * (1 + np.abs(Tr).max()))


@pytest.mark.parametrize("path", [4, 3])
@pytest.mark.parametrize("precision", [B.FP64, B.MIXED])
def test_column_blocked_solve_reaches_planted_optimum(precision, path):
    prob = PROBS["multi_block"]
    eps = 1e-6
    kw = dict(team=B.TEAM_GRID, spmv_path=path, precision=precision, eps=eps, max_iters=20000, cg_adapt=1e-2)
    work = B.Work(prob, **kw)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    A, b, c = prob["A"], prob["b"], prob["c"]
    pr = np.linalg.norm(A @ x + s - b) / (1 + np.linalg.norm(b))
    dr = np.linalg.norm(A.T @ y + c) / (1 + np.linalg.norm(c))
    assert max(pr, dr) <= eps * 1.01
    pstar = c @ prob["xstar"]
    assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))
    # the column-blocked products are deterministic: a repeat solve is identical
    x2, _, _, info2 = work.solve()
    np.testing.assert_array_equal(x, x2)
    assert info2["iters"] == info["iters"]
