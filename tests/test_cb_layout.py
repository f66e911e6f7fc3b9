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


def _check_tile(A, seed, **kw):
    A = sp.csr_matrix(A)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.shape[1])
    y, st = B.tile_layout_check(A, x, **kw)
    assert st["column_blocks"] > 0, st
    assert st["violations"] == 0, st
    # each tile's row sum, then the ncb partials in block order
    k = int(np.diff(A.indptr).max(initial=0)) + st["column_blocks"]
    bound = _gamma(k + 1) * (abs(A) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - A @ x) <= bound)
    return st


@pytest.mark.parametrize("elem_bytes", [4, 8])
@pytest.mark.parametrize("vectors", [1, 2])
def test_tiles_random_matrix(elem_bytes, vectors):
    """Two-dimensional tiles: several row and column blocks, several chunks per tile."""
    rng = np.random.default_rng(13)
    A = W.random_pattern(rng, 40000, 30001, 600_000)
    smem = 72000 if elem_bytes == 4 else 110000  # small enough that tiles need several stages
    st = _check_tile(A, 1, elem_bytes=elem_bytes, vectors=vectors, smem_bytes=smem)
    assert st["row_blocks"] * st["column_blocks"] <= 152 and st["smem_bytes"] <= smem
    assert st["chunks"] > 152  # tiles span more than one stage
    assert st["entries"] <= 1.6 * A.nnz


def test_tiles_skewed_and_empty_lines():
    """Dense rows and columns, empty rows and columns: a split whose slices fit a stage is found."""
    rng = np.random.default_rng(15)
    m, n = 30000, 20001
    A = W.random_pattern(rng, m, n, 200_000).tolil()
    for i in rng.choice(m, 3, replace=False):
        cols = rng.choice(n, 2000, replace=False)
        A[i, cols] = rng.standard_normal(2000)
    for j in rng.choice(n, 3, replace=False):
        rows = rng.choice(m, 3000, replace=False)
        A[rows, j] = rng.standard_normal((3000, 1))
    A = sp.csr_matrix(A)
    keep_r = np.ones(m)
    keep_r[rng.choice(m, 500, replace=False)] = 0
    keep_c = np.ones(n)
    keep_c[rng.choice(n, 400, replace=False)] = 0
    A = sp.csr_matrix(sp.diags(keep_r) @ A @ sp.diags(keep_c))
    A.eliminate_zeros()
    for eb in (4, 8):
        _check_tile(A, 2, elem_bytes=eb, vectors=2)


@pytest.mark.parametrize("ctas,warps", [(1, 1), (6, 3), (152, 15), (152, 7)])
def test_tiles_team_shapes(ctas, warps):
    rng = np.random.default_rng(ctas * 7 + warps)
    A = W.random_pattern(rng, 9000, 7001, 90_000)
    _check_tile(A, 4, ctas=ctas, compute_warps=warps, elem_bytes=4, vectors=1)


def test_tiles_c2_shape_split():
    """At the 1e7-nonzero benchmark shape (here 1/20 of the entries, same
    rows and columns) the FP32 split keeps every vector slice and row array
    in shared memory: A (200000 x 100000) and its transpose both split over
    all 152 CTAs."""
    rng = np.random.default_rng(17)
    A = W.random_pattern(rng, 200_000, 100_000, 500_000)
    for M, nv in ((A, 1), (sp.csr_matrix(A.T), 2)):
        st = _check_tile(M, 5, elem_bytes=4, vectors=nv)
        assert st["row_blocks"] * st["column_blocks"] == 152


def test_invalid_arguments_rejected():
    A = sp.csr_matrix(np.eye(4))
    with pytest.raises(B.SCSError):
        B.cb_layout_check(A, np.ones(4), elem_bytes=2)
    with pytest.raises(B.SCSError):
        B.cb_layout_check(A, np.ones(4), vectors=3)
    with pytest.raises(B.SCSError):
        B.tile_layout_check(A, np.ones(4), elem_bytes=2)
