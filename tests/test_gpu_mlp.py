"""GPU checks of the warm-start MLP kernels against the FP64 numpy oracle.

The GPU runs the GEMMs in BF16 (8-bit mantissa) with FP32 accumulation, so
gradients agree with the FP64 oracle only up to the BF16 rounding of inputs,
weights and activations, about 2^-9 relative per element.  The first layer's
weight gradient carries three such roundings (dh2, dh1 and the inputs) and is
a sum over the batch with cancellation, which amplifies the relative error of
the sum above the per-term error; measured 3-6% in Frobenius norm at cosine
>= 0.998.  The bounds used: relative error <= 0.1 and cosine >= 0.995 per
parameter block, loss and outputs within 2%.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1903_06477_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _blocks(dims):
    din, dh, dout = dims
    sizes = [dh * din, dh, dh * dh, dh, dout * dh, dout]
    return np.cumsum([0] + sizes)


@pytest.mark.parametrize("gemm", [B.GEMM_MMA, B.GEMM_TCGEN05])
@pytest.mark.parametrize("dims,batch", [((40, 64, 50), 32), ((300, 128, 1001), 77), ((2000, 256, 2203), 256),
                                        ((2000, 1024, 22004), 256)])  # the last: the warm-start network itself
def test_gradients_vs_oracle(dims, batch, gemm):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(sum(dims))
    net = B.MLP(*dims, max_batch=max(batch, 64), seed=3, gemm=gemm)
    X = rng.standard_normal((batch, dims[0])).astype(np.float32)
    T = rng.standard_normal((batch, dims[2])).astype(np.float32)
    Xd = torch.as_tensor(X, device="cuda")
    Td = torch.as_tensor(T, device="cuda")
    net.fit_normalization(Xd, Td)
    g = torch.empty(net.num_params, dtype=torch.float32, device="cuda")
    loss = net.gradients(Xd, Td, g)
    theta = net.get_params()
    norm = (X.astype(np.float64).mean(0), X.astype(np.float64).std(0), T.astype(np.float64).mean(0),
            T.astype(np.float64).std(0))
    ref_loss, ref_g, ref_y = M.loss_and_grad(theta, X, T, dims, norm)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    gg = g.cpu().numpy().astype(np.float64)
    b = _blocks(dims)
    for k in range(6):
        a, r = gg[b[k]:b[k + 1]], ref_g[b[k]:b[k + 1]]
        rel = np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)
        cos = a @ r / max(np.linalg.norm(a) * np.linalg.norm(r), 1e-30)
        assert rel <= 0.1 and cos >= 0.995, (k, rel, cos)
    Y = torch.empty(batch, dims[2], dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    yy = Y.cpu().numpy()
    assert np.linalg.norm(yy - ref_y) <= 2e-2 * np.linalg.norm(ref_y)


def test_training_reduces_loss_and_params_roundtrip():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    dims = (64, 128, 96)
    Wt = rng.standard_normal((96, 64)) / 8
    X = rng.standard_normal((2048, 64)).astype(np.float32)
    T = (np.tanh(X @ Wt.T) + 0.01 * rng.standard_normal((2048, 96))).astype(np.float32)
    Xd, Td = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    net = B.MLP(*dims, max_batch=256, seed=1)
    net.fit_normalization(Xd, Td)
    first = None
    for epoch in range(30):
        for i in range(0, 2048, 256):
            l = net.train_step(Xd[i:i + 256], Td[i:i + 256], 1e-3)
            first = l if first is None else first
    assert l < 0.2 * first, (first, l)
    p = net.get_params()
    net2 = B.MLP(*dims, max_batch=256, seed=77)
    net2.set_params(p)
    net2.fit_normalization(Xd, Td)
    Y1 = torch.empty(256, 96, device="cuda")
    Y2 = torch.empty(256, 96, device="cuda")
    net.forward(Xd[:256], Y1)
    net2.forward(Xd[:256], Y2)
    torch.testing.assert_close(Y1, Y2, rtol=0, atol=0)
