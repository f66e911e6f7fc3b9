"""Host-side checks of the column-blocked sparse layout (no GPU needed).

The grid team's column-blocked layout is built on the host.  scs_cb_layout_check
builds it, verifies its invariants (block widths, shared-memory budget and
alignment, segment metadata, distinct rows per segment, the ring's
look-ahead ranges, every stored column inside its block) and replays
y = A x in FP64 walking the layout exactly as the device loop does; the
result must equal the CSR product up to FP64 summation order:
|y - A x| <= gamma_k |A||x| with k the longest row, gamma_k = k u / (1 - k u).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1903_06477_gb300 import binding as B
from paper_1903_06477_gb300 import workloads as W

U64 = 2.0 ** -53


def _gamma(k):
    return k * U64 / (1 - k * U64)


def _check(A, seed, **kw):
    A = sp.csr_matrix(A)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.shape[1])
    y, st = B.cb_layout_check(A, x, **kw)
    assert st["column_blocks"] > 0, st
    assert st["violations"] == 0, st
    k = int(np.diff(A.indptr).max(initial=0))
    bound = _gamma(k + 1) * (abs(A) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - A @ x) <= bound)
    return st


@pytest.mark.parametrize("elem_bytes", [4, 8])
@pytest.mark.parametrize("vectors", [1, 2])
def test_random_matrix_several_blocks(elem_bytes, vectors):
    rng = np.random.default_rng(3)
    A = W.random_pattern(rng, 20000, 30001, 300_000)
    st = _check(A, 1, elem_bytes=elem_bytes, vectors=vectors)
    assert st["column_blocks"] >= 2  # the vector does not fit one stage
    assert st["entries"] <= 1.5 * A.nnz  # padding stays moderate


def test_skewed_rows_and_columns_and_empty_lines():
    rng = np.random.default_rng(5)
    m, n = 12000, 9001
    A = W.random_pattern(rng, m, n, 80_000).tolil()
    for i in rng.choice(m, 4, replace=False):
        cols = rng.choice(n, 3000, replace=False)
        A[i, cols] = rng.standard_normal(3000)
    for j in rng.choice(n, 3, replace=False):
        rows = rng.choice(m, 2000, replace=False)
        A[rows, j] = rng.standard_normal((2000, 1))
    A = sp.csr_matrix(A)
    keep_r = np.ones(m)
    keep_r[rng.choice(m, 300, replace=False)] = 0
    keep_c = np.ones(n)
    keep_c[rng.choice(n, 200, replace=False)] = 0
    A = sp.diags(keep_r) @ A @ sp.diags(keep_c)
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    for eb in (4, 8):
        _check(A, 2, elem_bytes=eb, vectors=2)


def test_fewer_rows_than_ctas_and_tiny_blocks():
    rng = np.random.default_rng(7)
    A = W.random_pattern(rng, 53, 37, 500)
    st = _check(A, 3, elem_bytes=8, vectors=2)
    assert st["column_blocks"] == 1


@pytest.mark.parametrize("ctas,warps", [(1, 1), (4, 3), (152, 15), (152, 7)])
def test_team_shapes(ctas, warps):
    rng = np.random.default_rng(ctas + warps)
    A = W.random_pattern(rng, 5000, 7001, 60_000)
    _check(A, 4, ctas=ctas, compute_warps=warps, elem_bytes=4, vectors=1)


def test_layout_that_does_not_fit_is_reported():
    # one CTA would need partial sums for 70000 rows: more than 16-bit row
    # indices and the shared memory allow, so the solver keeps sliced ELL
    rng = np.random.default_rng(9)
    A = W.random_pattern(rng, 70000, 1000, 70_000)
    y, st = B.cb_layout_check(A, np.ones(1000), ctas=1, compute_warps=15)
    assert st["column_blocks"] == 0


def test_invalid_arguments_rejected():
    A = sp.csr_matrix(np.eye(4))
    with pytest.raises(B.SCSError):
        B.cb_layout_check(A, np.ones(4), elem_bytes=2)
    with pytest.raises(B.SCSError):
        B.cb_layout_check(A, np.ones(4), vectors=3)
