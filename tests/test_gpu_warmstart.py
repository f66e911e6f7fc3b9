"""GPU tests of warm starts, the cold-start fallback, shared-matrix batches and
the learned warm start (MLP trained by the library's kernels on solutions of
the library's own batched solver)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import binding as B
from paper_1903_06477_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _kkt(prob, x, y, s):
    A, b, c = prob["A"], prob["b"], prob["c"]
    pr = np.linalg.norm(A @ x + s - b) / (1 + np.linalg.norm(b))
    dr = np.linalg.norm(A.T @ y + c) / (1 + np.linalg.norm(c))
    cx, by = c @ x, b @ y
    return max(pr, dr, abs(cx + by) / (1 + abs(cx) + abs(by)))


def test_warm_start_and_fallback():
    prob = W.planted(seed=51, n=200, l=150, soc=[10] * 5, nnz=3000)
    eps = 1e-6
    w = B.Work(prob, eps=eps, max_iters=20000, warm_fallback=20)
    x, y, s, info = w.solve()
    assert info["status"] == B.SOLVED
    u = w.get_u()
    # warm from the solution: done almost at once, no fallback
    w.set_warm(u)
    _, _, _, i2 = w.solve()
    assert i2["status"] == B.SOLVED and i2["iters"] <= 3 and i2["warm_fallback_taken"] == 0
    # warm from a bad point: the fallback restarts cold and still solves
    w.set_warm(np.random.default_rng(0).standard_normal(w.N) * 1e4)
    x3, y3, s3, i3 = w.solve()
    assert i3["status"] == B.SOLVED and i3["warm_fallback_taken"] == 1
    assert _kkt(prob, x3, y3, s3) <= eps * 1.01


@pytest.mark.parametrize("precision", [B.FP64, B.MIXED])
def test_shared_batch_matches_single_solves(precision):
    F = W.lasso_family_matrix(seed=3, p=40, nvar=90, density=0.1)
    gs = [W.lasso_family_rhs(F, seed=700 + i) for i in range(24)]
    prob0 = W.lasso(F=F, g=gs[0])
    bcs = [W.lasso_family_bc(F, g) for g in gs]
    eps = 1e-6
    batch = B.Batch(shared=(prob0, [b for b, _ in bcs], [c for _, c in bcs]), precision=precision, eps=eps,
                    max_iters=20000)
    xs, ys, ss, infos = batch.solve()
    for g, (b, c), x, y, s, info in zip(gs, bcs, xs, ys, ss, infos):
        p = dict(prob0, b=b, c=c)
        assert info["status"] == B.SOLVED
        assert _kkt(p, x, y, s) <= eps * 1.01
        ref = O.Oracle(p, eps=eps, max_iters=20000).solve()
        assert abs(info["pobj"] - ref["info"].pobj) <= 10 * eps * (1 + abs(ref["info"].pobj))


def test_learned_warm_start_gains_iterations():
    """A parametric LASSO family whose solutions vary smoothly with g (fixed
    support, +-10% amplitudes): the network trained on 1536 solutions by the
    library's kernels cuts the median outer-iteration count on 64 held-out
    instances below 80% of the cold start's (the oracle with an even simpler,
    linear predictor goes from 166 to 75), and every warm-started solve still
    meets eps (the cold start is the fallback).  With a random support per
    instance the solution map is a sparse-recovery problem that no network of
    this size learns from this much data; that case is measured by the C5
    benchmark."""
    torch = pytest.importorskip("torch")
    F = W.lasso_family_matrix(seed=4, p=64, nvar=160, density=0.1)
    eps = 1e-5
    kw = dict(direction=B.DIR_RB, mem=10, c0=0.1, precision=B.FP64, eps=eps, max_iters=20000, cg_adapt=1e-2,
              warm_fallback=50)

    def solve(gs, warm=None):
        bcs = [W.lasso_family_bc(F, g) for g in gs]
        prob0 = W.lasso(F=F, g=gs[0])
        batch = B.Batch(shared=(prob0, [b for b, _ in bcs], [c for _, c in bcs]), **kw)
        if warm is not None:
            batch.set_warm(warm)
        xs, ys, ss, infos = batch.solve()
        return prob0, bcs, xs, ys, ss, infos

    gtr = [W.lasso_family_rhs_smooth(F, seed=10_000 + i, base_seed=4) for i in range(1536)]
    _, _, xs, ys, ss, infos = solve(gtr)
    assert all(i["status"] == B.SOLVED for i in infos)
    U = np.stack([np.concatenate([x, y + s, [1.0]]) for x, y, s in zip(xs, ys, ss)]).astype(np.float32)
    G = np.stack(gtr).astype(np.float32)
    Xd, Ud = torch.as_tensor(G, device="cuda"), torch.as_tensor(U, device="cuda")
    net = B.MLP(G.shape[1], 256, U.shape[1], max_batch=256, seed=5)
    net.fit_normalization(Xd, Ud)
    lr = 2e-3
    for ep in range(60):
        perm = torch.randperm(len(G), device="cuda")
        for i in range(0, len(G), 256):
            idx = perm[i:i + 256]
            net.train_step(Xd[idx].contiguous(), Ud[idx].contiguous(), lr)
        lr *= 0.96
    gte = [W.lasso_family_rhs_smooth(F, seed=90_000 + j, base_seed=4) for j in range(64)]
    Xt = torch.as_tensor(np.stack(gte).astype(np.float32), device="cuda")
    Yt = torch.empty(64, U.shape[1], device="cuda")
    net.forward(Xt, Yt)
    warm = [row.astype(np.float64) for row in Yt.cpu().numpy()]
    for w in warm:
        w[-1] = 1.0
    prob0, bcs, _, _, _, cold = solve(gte)
    _, _, xs, ys, ss, hot = solve(gte, warm)
    for (b, c), x, y, s, info in zip(bcs, xs, ys, ss, hot):
        assert info["status"] == B.SOLVED
        assert _kkt(dict(prob0, b=b, c=c), x, y, s) <= eps * 1.01
    it_cold = np.median([i["iters"] for i in cold])
    it_hot = np.median([i["iters"] for i in hot])
    assert it_hot < 0.8 * it_cold, (it_cold, it_hot)
