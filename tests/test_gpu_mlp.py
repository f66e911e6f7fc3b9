"""GPU checks of the warm-start MLP kernels, each on its own actual inputs.

Every stage of the network is read back through scs_mlp_read and compared
element by element with an FP64 evaluation of the same formula on the same
BF16-rounded operands the GPU used, within the bound the arithmetic allows:
  - products of BF16 values are exact in FP32, so a GEMM of depth K differs
    from the FP64 sum by at most gamma_K * sum|a b| (FP32 accumulation; the
    bound below doubles it for the tensor cores' accumulation order), plus
    one FP32 rounding for the bias;
  - a value stored in BF16 adds one rounding of at most 2^-8 relative;
  - elementwise FP32 kernels (normalisation, loss gradient, column sums,
    denormalisation, Adam) are checked against FP64 within a few units of
    FP32 rounding of the quantities involved;
  - BF16 copies of FP32 values (weights, dy, dh) are checked bit for bit
    against round-to-nearest-even.
The Adam update is compared with the FP64 oracle's step (Kingma and Ba,
with bias corrections) from the GPU's own parameters, gradient and moments,
for two consecutive steps.  A separate loose end-to-end comparison with the
pure FP64 oracle (no BF16 anywhere) checks the composition.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1903_06477_gb300 import binding as B

pytestmark = pytest.mark.gpu

U = 2.0 ** -24  # FP32 unit roundoff
UB = 2.0 ** -8  # BF16 unit roundoff (8 significant bits, round to nearest)


def bf16(x):
    """FP32 -> BF16 round to nearest, ties to even (finite values), as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).reshape(np.shape(x))


def _blocks(dims):
    din, dh, dout = dims
    sizes = [dh * din, dh, dh * dh, dh, dout * dh, dout]
    return np.cumsum([0] + sizes)


def _split(theta, dims):
    din, dh, dout = dims
    b = _blocks(dims)
    shapes = [(dh, din), (dh,), (dh, dh), (dh,), (dout, dh), (dout,)]
    return [np.asarray(theta[b[k]:b[k + 1]], np.float64).reshape(shapes[k]) for k in range(6)]


def check_gemm(name, out, A, Bt, bias=None, relu=False, mask=None, bf16_out=False):
    """out ~ op(A @ Bt^T + bias) with A, Bt exact (BF16 values) in FP64."""
    A = np.asarray(A, np.float64)
    Bt = np.asarray(Bt, np.float64)
    z = A @ Bt.T
    S = np.abs(A) @ np.abs(Bt).T
    if bias is not None:
        z = z + bias
        S = S + np.abs(bias)
    keep = np.ones_like(z, dtype=bool) if mask is None else (np.asarray(mask) > 0)
    ref = np.where(keep, np.maximum(z, 0.0) if relu else z, 0.0)
    K = A.shape[1]
    bound = 2.0 * (K + 2) * U * S * keep + 2 * U * np.abs(ref) + 1e-30
    if bf16_out:
        bound = bound + UB * np.abs(ref) * 1.01
    err = np.abs(np.asarray(out, np.float64) - ref)
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert (err <= bound).all(), (name, worst, err[worst], bound[worst], ref[worst])


def check_colsum(name, out, D):
    D = np.asarray(D, np.float64)
    ref = D.sum(0)
    bound = (D.shape[0] + 1) * U * np.abs(D).sum(0) + 1e-30
    err = np.abs(np.asarray(out, np.float64).ravel() - ref)
    assert (err <= bound).all(), (name, np.argmax(err / bound))


def run_stages(net, dims, X, T, gemm):
    """gradients() on one batch, then every stage checked from its actual inputs; returns (loss, grad)."""
    torch = pytest.importorskip("torch")
    din, dh, dout = dims
    Bn = X.shape[0]
    Xd, Td = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    g = torch.empty(net.num_params, dtype=torch.float32, device="cuda")
    loss = net.gradients(Xd, Td, g)
    theta = net.read("params").ravel()
    W1, b1, W2, b2, W3, b3 = _split(theta, dims)
    r = {k: net.read(k).astype(np.float64) for k in B.MLP_BUFFERS if k not in ("params", "adam_m", "adam_v")}
    # normalisation statistics (two-pass FP64 on the device, stored in FP32)
    X64, T64 = X.astype(np.float64), T.astype(np.float64)
    for nm, ref in (("in_mean", X64.mean(0)), ("in_std", X64.std(0)), ("out_mean", T64.mean(0)),
                    ("out_std", T64.std(0))):
        ref32 = np.where(ref >= 1e-6, ref, 1.0) if nm.endswith("std") else ref
        ref32 = ref32.astype(np.float32).astype(np.float64)
        assert (np.abs(r[nm].ravel() - ref32) <= np.spacing(np.abs(ref32).astype(np.float32))).all(), nm
    mean_i, sd_i = X64.mean(0), X64.std(0)
    mean_o, sd_o = T64.mean(0), T64.std(0)
    # BF16 weight copies, bit for bit, and the transposed copies of the backward pass
    for nm, W in (("w1", W1), ("w2", W2), ("w3", W3)):
        assert np.array_equal(r[nm], bf16(W.astype(np.float32)).astype(np.float64)), nm
    assert np.array_equal(r["w2t"], r["w2"].T) and np.array_equal(r["w3t"], r["w3"].T)
    # normalised input: (x - mean) * (1/std) in FP32, then BF16
    ref = (X64 - mean_i) / sd_i
    bound = UB * np.abs(ref) * 1.01 + 4 * U * (np.abs(ref) + np.abs(mean_i / sd_i)) + 1e-30
    assert (np.abs(r["xn"] - ref) <= bound).all(), "normalize_to_bf16"
    # forward GEMMs with bias and ReLU
    check_gemm("h1", r["h1"], r["xn"], r["w1"], bias=b1, relu=True, bf16_out=True)
    check_gemm("h2", r["h2"], r["h1"], r["w2"], bias=b2, relu=True, bf16_out=True)
    check_gemm("y", r["y"], r["h2"], r["w3"], bias=b3)
    # loss and its gradient
    tn = (T64 - mean_o) / sd_o
    diff = r["y"] - tn
    ref_loss = 0.5 * np.mean(diff ** 2)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss + 1e-30, (loss, ref_loss)
    scale = 1.0 / (Bn * dout)
    ref = diff * scale
    bound = 6 * U * (np.abs(r["y"]) + np.abs(tn) + np.abs(mean_o / sd_o)) * scale + 1e-38
    assert (np.abs(r["dy"] - ref) <= bound).all(), "loss_grad"
    assert np.array_equal(r["dy16"], bf16(r["dy"].astype(np.float32)).astype(np.float64)), "dy16"
    # backward GEMMs (transposed weights, ReLU masks of the forward activations)
    check_gemm("dh2", r["dh2"], r["dy16"], r["w3t"], mask=r["h2"])
    assert np.array_equal(r["dh2_16"], bf16(r["dh2"].astype(np.float32)).astype(np.float64)), "dh2_16"
    check_gemm("dh1", r["dh1"], r["dh2_16"], r["w2t"], mask=r["h1"])
    assert np.array_equal(r["dh1_16"], bf16(r["dh1"].astype(np.float32)).astype(np.float64)), "dh1_16"
    # parameter gradients: weight GEMMs over the batch, bias column sums
    gg = g.cpu().numpy().astype(np.float64)
    assert np.array_equal(gg, r["grad"].ravel())
    gW1, gb1, gW2, gb2, gW3, gb3 = _split(gg, dims)
    check_gemm("gW3", gW3, r["dy16"].T, r["h2"].T)
    check_colsum("gb3", gb3, r["dy"])
    check_gemm("gW2", gW2, r["dh2_16"].T, r["h1"].T)
    check_colsum("gb2", gb2, r["dh2"])
    check_gemm("gW1", gW1, r["dh1_16"].T, r["xn"].T)
    check_colsum("gb1", gb1, r["dh1"])
    # denormalised forward output
    Y = torch.empty(Bn, dout, dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    yy = Y.cpu().numpy().astype(np.float64)
    y_again = net.read("y").astype(np.float64)
    ref = y_again * r["out_std"] + r["out_mean"]
    assert (np.abs(yy - ref) <= 2 * U * (np.abs(y_again * r["out_std"]) + np.abs(r["out_mean"])) + 1e-30).all()
    return loss, gg, theta


@pytest.mark.parametrize("gemm", [B.GEMM_MMA, B.GEMM_TCGEN05])
@pytest.mark.parametrize("dims,batch", [((40, 64, 50), 32), ((300, 128, 1001), 77), ((2000, 256, 2203), 256),
                                        ((2000, 1024, 22004), 256)])  # the last: the warm-start network itself
def test_every_stage_on_its_own_inputs(dims, batch, gemm):
    rng = np.random.default_rng(sum(dims))
    net = B.MLP(*dims, max_batch=max(batch, 64), seed=3, gemm=gemm)
    X = rng.standard_normal((batch, dims[0])).astype(np.float32)
    T = rng.standard_normal((batch, dims[2])).astype(np.float32)
    torch = pytest.importorskip("torch")
    net.fit_normalization(torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda"))
    loss, gg, theta = run_stages(net, dims, X, T, gemm)
    # loose end-to-end check against the pure FP64 oracle (no BF16 rounding at all)
    X64, T64 = X.astype(np.float64), T.astype(np.float64)
    norm = (X64.mean(0), X64.std(0), T64.mean(0), T64.std(0))
    ref_loss, ref_g, _ = M.loss_and_grad(theta, X, T, dims, norm)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    b = _blocks(dims)
    for k in range(6):
        a, rr = gg[b[k]:b[k + 1]], ref_g[b[k]:b[k + 1]]
        assert a @ rr >= 0.99 * np.linalg.norm(a) * np.linalg.norm(rr), k
    net.close()


def test_adam_steps_match_oracle():
    """Two train steps: each parameter update against the oracle's Adam step
    from the GPU's own parameters, gradient and moments before the step."""
    torch = pytest.importorskip("torch")
    dims, batch = (300, 128, 1001), 77
    rng = np.random.default_rng(17)
    X = rng.standard_normal((batch, dims[0])).astype(np.float32)
    T = rng.standard_normal((batch, dims[2])).astype(np.float32)
    Xd, Td = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    net = B.MLP(*dims, max_batch=128, seed=5)
    net.fit_normalization(Xd, Td)
    lr = 2.0 ** -10  # exactly representable in FP32
    th = net.read("params").ravel().astype(np.float64)
    m = net.read("adam_m").ravel().astype(np.float64)
    v = net.read("adam_v").ravel().astype(np.float64)
    assert not m.any() and not v.any()
    for t in (1, 2):
        net.train_step(Xd, Td, lr)
        g = net.read("grad").ravel().astype(np.float64)
        th1 = net.read("params").ravel().astype(np.float64)
        m1 = net.read("adam_m").ravel().astype(np.float64)
        v1 = net.read("adam_v").ravel().astype(np.float64)
        th_r, m_r, v_r = M.adam_step(th, g, m, v, t, lr)
        assert (np.abs(m1 - m_r) <= 4 * U * (np.abs(m) + np.abs(g)) + 1e-45).all(), ("m", t)
        assert (np.abs(v1 - v_r) <= 6 * U * (np.abs(v) + g * g) + 1e-45).all(), ("v", t)
        # theta: the final FP32 operations (a few roundings of the step and one of theta), plus
        # the first-order effect of the moments' own deviations (each checked just above)
        step = th - th_r
        b1c, b2c = 1 - 0.9 ** t, 1 - 0.999 ** t
        den = np.sqrt(v_r / b2c) + 1e-8
        dm, dv = np.abs(m1 - m_r), np.abs(v1 - v_r)
        bound = (U * np.abs(th_r) + 10 * U * np.abs(step) + lr * (dm + 2 * U * np.abs(m_r)) / (b1c * den)
                 + np.abs(step) * dv / (2 * np.maximum(v_r, 1e-300)) + 1e-45)
        assert (np.abs(th1 - th_r) <= bound).all(), ("theta", t, np.max(np.abs(th1 - th_r) / bound))
        assert np.abs(step).max() > 0
        # the BF16 weight copies follow the updated parameters
        W1, _, W2, _, W3, _ = _split(th1, dims)
        for nm, W in (("w1", W1), ("w2", W2), ("w3", W3)):
            assert np.array_equal(net.read(nm).astype(np.float64), bf16(W.astype(np.float32)).astype(np.float64))
        assert np.array_equal(net.read("w2t"), net.read("w2").T) and np.array_equal(net.read("w3t"), net.read("w3").T)
        th, m, v = th1, m1, v1
    net.close()


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
