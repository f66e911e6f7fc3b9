"""GPU parity of the MLP's two GEMM kernels (C = A B^T, BF16 operands, FP32
accumulation): the warp-level MMA kernel and the tcgen05 kernel with its
accumulator in tensor memory.

Reference: the same BF16 values multiplied in FP64 on the host.  The
products of two BF16 numbers are exact in FP32, so the only error is the
FP32 accumulation over K terms: |C - AB^T| <= gamma_K (|A||B|^T) with
gamma_K ~ K u, u = 2^-24; the test allows 2 K u to cover an accumulator
that truncates instead of rounding.  Shapes cover a single tile, tails in
M, N and K (K not a multiple of 8 reads a partial 16-byte chunk), K = 0,
several K blocks, and the network's own products.
"""
import numpy as np
import pytest

from paper_1903_06477_gb300 import binding as B

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (7, 129, 9), (128, 128, 64), (130, 200, 72), (300, 260, 0), (129, 257, 1000),
          (256, 1024, 2000), (256, 22004, 1024), (1024, 2000, 256), (256, 1024, 22004)]


def _operand(torch, rng, rows, K):
    ld = (K + 7) // 8 * 8 if K > 0 else 8
    full = torch.zeros(rows, ld, dtype=torch.bfloat16, device="cuda")
    if K > 0:
        full[:, :K] = torch.as_tensor(rng.standard_normal((rows, K)).astype(np.float32), device="cuda")
    return full[:, :K] if K > 0 else full[:, :0]


@pytest.mark.parametrize("impl", [B.GEMM_MMA, B.GEMM_TCGEN05])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_nt_matches_fp64(M, N, K, impl):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = _operand(torch, rng, M, K)
    Bm = _operand(torch, rng, N, K)
    C = B.gemm_nt(A, Bm, impl=impl)
    a = A.float().cpu().numpy().astype(np.float64)
    b = Bm.float().cpu().numpy().astype(np.float64)
    ref = a @ b.T
    bound = 2 * max(K, 1) * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(C.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= bound), (float(err.max()), float((err - bound).max()))


def test_gemm_nt_rejects_bad_strides():
    torch = pytest.importorskip("torch")
    A = torch.zeros(4, 12, dtype=torch.bfloat16, device="cuda")  # row stride 12: not a multiple of 8
    with pytest.raises(B.SCSError):
        B.gemm_nt(A, A, impl=B.GEMM_TCGEN05)
