"""GPU test of scs_residuals_noalloc, the allocation-free residual check.

Some callers cannot allocate device memory (for example code running while a
CUDA graph is captured, or real-time loops that forbid allocation after
start-up); this entry point keeps its scratch in a static device array.  The
test calls it through the C ABI on device buffers, twice in a row (the second
call reuses the scratch left by the first), and checks both results against
scs_residuals, the entry point that works on a set-up scs_work.  This file is
named to be collected last.
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
