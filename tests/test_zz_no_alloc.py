"""GPU test of scs_residuals_noalloc, the allocation-free residual check.

Some callers cannot allocate device memory (real-time loops that forbid
allocation after start-up, because cudaMalloc may block and synchronise the
device, or hosts whose device memory belongs to another allocator); this entry
point keeps its scratch in a static device array.  The test calls it through
the C ABI on device buffers, twice in a row (the second call reuses the
scratch left by the first), and checks both results against scs_residuals, the
entry point that works on a set-up scs_work.  This file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1903_06477_gb300 import binding as B
from paper_1903_06477_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_noalloc_matches_work_entry_twice():
    torch = pytest.importorskip("torch")
    L = B.lib()
    prob = W.planted(seed=31, n=3000, l=2500, soc=[20] * 50, f=10, nnz=60000)
    work = B.Work(prob, eps=1e-6, max_iters=20000)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED
    A = prob["A"]
    m, n = A.shape
    Ap = _dev(torch, A.indptr.astype(np.int64), torch.int64)
    Ai = _dev(torch, A.indices.astype(np.int32), torch.int32)
    Ax = _dev(torch, A.data, torch.float64)
    b = _dev(torch, prob["b"], torch.float64)
    c = _dev(torch, prob["c"], torch.float64)
    rng = np.random.default_rng(5)
    candidates = [(x, y, s), (rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m))]
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for xc, yc, sc in candidates:
        ref = work.residuals(xc, yc, sc)
        xd, yd, sd = (_dev(torch, v, torch.float64) for v in (xc, yc, sc))
        for _ in range(2):
            out.fill_(float("nan"))
            rc = L.scs_residuals_noalloc(m, n, Ap.data_ptr(), Ai.data_ptr(), Ax.data_ptr(), b.data_ptr(),
                                         c.data_ptr(), xd.data_ptr(), yd.data_ptr(), sd.data_ptr(),
                                         out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == B.SCS_OK, B.last_error()
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-9, atol=1e-12)


def test_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    L = B.lib()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    rc = L.scs_residuals_noalloc(4, (1 << 20) + 1, p, p, p, p, p, p, p, p, p, None)
    assert rc == B.SCS_EINVAL
    assert "1048576" in B.last_error()


def test_noalloc_bad_column_index_gives_nan():
    """A column index outside [0, n) is skipped by the kernel's bounds check
    (nothing out of range is read or written) and all three outputs are NaN;
    a correct call right after gives finite results again."""
    torch = pytest.importorskip("torch")
    L = B.lib()
    m, n = 3, 4
    Ap = _dev(torch, np.array([0, 2, 3, 4], np.int64), torch.int64)
    Ai_bad = _dev(torch, np.array([0, 4, 1, 3], np.int32), torch.int32)  # 4 == n is out of range
    Ai_ok = _dev(torch, np.array([0, 2, 1, 3], np.int32), torch.int32)
    Ax = _dev(torch, np.array([1.0, 2.0, 3.0, 4.0]), torch.float64)
    b, y, s = (_dev(torch, np.ones(m), torch.float64) for _ in range(3))
    c, x = (_dev(torch, np.ones(n), torch.float64) for _ in range(2))
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = [Ap.data_ptr(), None, Ax.data_ptr(), b.data_ptr(), c.data_ptr(), x.data_ptr(), y.data_ptr(),
            s.data_ptr(), out.data_ptr(), stream]
    args[1] = Ai_bad.data_ptr()
    assert L.scs_residuals_noalloc(m, n, *args) == B.SCS_OK, B.last_error()
    torch.cuda.synchronize()
    assert np.isnan(out.cpu().numpy()).all()
    args[1] = Ai_ok.data_ptr()
    assert L.scs_residuals_noalloc(m, n, *args) == B.SCS_OK, B.last_error()
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()
