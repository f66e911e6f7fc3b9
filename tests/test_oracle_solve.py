"""Pins for Algorithm 1 (SuperSCS) and the whole-solve results of the oracle.

- KM limit: with d = 0 and K0 off, every step is K2 with rho = ||Ru||^2, i.e.
  the Krasnosel'skii-Mann iteration u+ = (1-lambda) u + lambda T u (Eq. km);
  compared with an independent 5-line loop over T.
- K0 path: with c0 so large that every step is K0, Algorithm 1 is the
  undamped quasi-Newton iteration u+ = u + d on R = I - T.  With Anderson
  directions that is Anderson acceleration of the fixed-point map T in
  Walker and Ni's form (window mem, least squares by numpy.linalg.lstsq);
  with restarted Broyden it is the Broyden iteration with Powell's theta
  safeguard carried out on a dense inverse-Jacobian estimate H.  Both are
  compared with the oracle's iterate after each of a dozen steps; the same
  path forced through K1 at alpha = 1 (c0 = 0, c1 = 1e300) must match too.
- Branch invariants: K1 steps satisfy ||Ru+|| <= c1 ||Ru||; K2 steps are
  Fejer monotone with respect to the planted fixed point.
- End results: planted optima (objective c^T x*), LASSO against an independent
  FISTA, and planted infeasible / unbounded certificates.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import workloads as W
from tests.helpers import check_in_cone, fista_lasso


def test_km_limit():
    prob = W.planted(seed=11, n=40, l=30, soc=[4, 4], f=2, nnz=500)
    for lam in (1.0, 1.5, 0.5):
        iters = 25
        orc = O.Oracle(prob, direction=O.DIR_NONE, c0=0.0, c1=0.99, lam=lam, max_iters=iters,
                       eps=1e-30, cg_rtol=1e-15, cg_max=10000)
        out = orc.solve()
        assert out["info"].k2 == iters and out["info"].k0 == 0 and out["info"].k1 == 0
        ref = O.Oracle(prob, cg_rtol=1e-15, cg_max=10000)
        u = np.zeros(orc.N)
        u[-1] = 1.0
        for _ in range(iters):
            Tu, _ = ref.apply_T(u)
            u = (1 - lam) * u + lam * Tu
        np.testing.assert_allclose(out["u"], u, atol=1e-9 * (1 + np.abs(u).max()))


def _k0_oracle_path(prob, direction, mem, iters, branch="K0", **extra):
    """The oracle's iterate after 1, 2, ..., iters steps of Algorithm 1 with
    every step forced to K0 (c0 = 1e300), or to K1 at alpha = 1 (c0 = 0,
    c1 = 1e300: the safeguard ||Ru|| <= r_safe then holds at every step).
    Both branches then take u+ = u + d and store the pair (d, Ru+ - Ru)."""
    path = []
    forced = dict(c0=1e300) if branch == "K0" else dict(c0=0.0, c1=1e300)
    for k in range(1, iters + 1):
        orc = O.Oracle(prob, direction=direction, mem=mem, max_iters=k, eps=1e-30,
                       cg_rtol=1e-15, cg_max=10000, **forced, **extra)
        out = orc.solve()
        info = out["info"]
        assert (info.k0, info.k1, info.k2, info.backtracks) == ((k, 0, 0, 0) if branch == "K0" else (0, k, 0, 0))
        path.append(out["u"])
        orc.close()
    return path


@pytest.mark.parametrize("kind", [O.DIR_AA, O.DIR_AA_QR])
@pytest.mark.parametrize("branch", ["K0", "K1"])
@pytest.mark.parametrize("mem", [1, 3, 5])
def test_k0_path_is_anderson_acceleration(mem, branch, kind):
    prob = W.planted(seed=21, n=40, l=30, soc=[4, 4], f=2, nnz=500)
    iters = 12
    path = _k0_oracle_path(prob, kind, mem, iters, branch=branch, aa_reg=1e-15)
    ref = O.Oracle(prob, cg_rtol=1e-15, cg_max=10000)
    # Anderson acceleration (Walker and Ni) of g = T: f = g(u) - u = -Ru,
    # u+ = g(u) - G gamma with gamma = argmin ||f - F gamma|| over the last
    # mem differences F (of f) and G (of g)
    u = np.zeros(ref.N)
    u[-1] = 1.0
    Tu, Ru = ref.apply_T(u)
    dF, dG = [], []
    for k in range(iters):
        f, g = -Ru, Tu
        if dF:
            F = np.array(dF[-mem:]).T
            G = np.array(dG[-mem:]).T
            gamma = np.linalg.lstsq(F, f, rcond=None)[0]
            u_new = g - G @ gamma
        else:
            u_new = g
        Tn, Rn = ref.apply_T(u_new)
        dF.append(-Rn - f)
        dG.append(Tn - g)
        u, Tu, Ru = u_new, Tn, Rn
        scale = 1 + np.abs(u).max()
        np.testing.assert_allclose(path[k], u, rtol=0, atol=1e-10 * scale, err_msg=f"step {k + 1}")


@pytest.mark.parametrize("branch", ["K0", "K1"])
@pytest.mark.parametrize("mem", [2, 4])
def test_k0_path_is_safeguarded_broyden(mem, branch):
    prob = W.planted(seed=22, n=30, l=24, soc=[4], f=1, nnz=300)
    iters, tb = 12, 0.1
    path = _k0_oracle_path(prob, O.DIR_RB, mem, iters, branch=branch, thetabar=tb)
    ref = O.Oracle(prob, cg_rtol=1e-15, cg_max=10000)
    N = ref.N
    u = np.zeros(N)
    u[-1] = 1.0
    _, Ru = ref.apply_T(u)
    H, stored = np.eye(N), 0
    for k in range(iters):
        if k > 0:
            # Broyden update of the inverse estimate with the pair (z, xi),
            # xi~ = (1 - theta) B z + theta xi (Powell), H B = I
            Hxi = H @ xi
            gam = Hxi @ z / (z @ z)
            th = 1.0 if abs(gam) >= tb else (1 - (1.0 if gam >= 0 else -1.0) * tb) / (1 - gam)
            Hxi_t = (1 - th) * z + th * Hxi
            Hn = H + np.outer(z - Hxi_t, z @ H) / (z @ Hxi_t)
            d = -Hn @ Ru
            if stored == mem:  # memory full: restart, the current pair is not kept
                H, stored = np.eye(N), 0
            else:
                H, stored = Hn, stored + 1
        else:
            d = -Ru
        u_new = u + d
        _, Rn = ref.apply_T(u_new)
        z, xi = d, Rn - Ru
        u, Ru = u_new, Rn
        scale = 1 + np.abs(u).max()
        np.testing.assert_allclose(path[k], u, rtol=0, atol=1e-10 * scale, err_msg=f"step {k + 1}")


@pytest.mark.parametrize("direction,mem", [(O.DIR_AA, 10), (O.DIR_RB, 10), (O.DIR_AA, 3)])
def test_branch_invariants_planted(direction, mem):
    prob = W.planted(seed=12, n=60, l=60, soc=[5, 5, 8], f=2, nnz=1000)
    ustar = np.concatenate([prob["xstar"], prob["ystar"] + prob["sstar"], [1.0]])
    c0 = 0.99 if direction == O.DIR_AA else 0.1
    orc = O.Oracle(prob, direction=direction, mem=mem, c0=c0, eps=1e-9, max_iters=3000, cg_rtol=1e-13)
    out = orc.solve(trace_cap=3000, ustar=ustar)
    tr, info = out["trace"], out["info"]
    assert info.status == O.SOLVED
    nRu, step, dist = tr["nRu"], tr["step"], tr["u_dist"]
    c1 = orc.settings["c1"]
    for k in range(len(step) - 1):
        if step[k] == 1:
            assert nRu[k + 1] <= c1 * nRu[k] * (1 + 1e-12) + 1e-14
    # K2: Fejer monotone w.r.t. a fixed point (projection on a separating hyperplane)
    prev = np.concatenate([[np.linalg.norm(np.r_[np.zeros(orc.N - 1), 1.0] - ustar)], dist[:-1]])
    k2 = step == 2
    assert np.all(dist[k2] <= prev[k2] * (1 + 1e-9) + 1e-9)
    assert info.k0 + info.k1 + info.k2 == info.iters


def test_every_branch_fires():
    seen = dict(k0=0, k1=0, k2=0, backtracks=0)
    probs = [W.lasso(seed=s) for s in range(2)] + [W.planted(seed=13, n=60, l=60, soc=[5, 5], nnz=900)]
    for prob in probs:
        for direction, c0 in ((O.DIR_AA, 0.99), (O.DIR_RB, 0.1)):
            out = O.Oracle(prob, direction=direction, mem=10, c0=c0, eps=1e-7, max_iters=4000).solve()
            for k in seen:
                seen[k] += getattr(out["info"], k)
    assert all(v > 0 for v in seen.values()), seen


def _kkt_checks(prob, out, eps):
    A, b, c = prob["A"], prob["b"], prob["c"]
    x, y, s = out["x"], out["y"], out["s"]
    info = out["info"]
    assert info.status == O.SOLVED
    assert max(info.pr, info.dr, info.gap) <= eps
    pr = np.linalg.norm(A @ x + s - b) / (1 + np.linalg.norm(b))
    dr = np.linalg.norm(A.T @ y + c) / (1 + np.linalg.norm(c))
    assert pr <= eps * 1.0001 and dr <= eps * 1.0001
    check_in_cone(prob, s, dual=False, tol=1e-9 * (1 + np.abs(s).max()))
    check_in_cone(prob, y, dual=True, tol=1e-9 * (1 + np.abs(y).max()))
    assert abs(y @ s) <= 1e-8 * (1 + np.abs(y).max() * np.abs(s).max() * len(s))


@pytest.mark.parametrize("direction", [O.DIR_AA, O.DIR_RB])
def test_lasso_c1_vs_fista(direction):
    prob = W.lasso(seed=0)
    eps = 1e-9
    c0 = 0.99 if direction == O.DIR_AA else 0.1
    out = O.Oracle(prob, direction=direction, mem=10, c0=c0, eps=eps, max_iters=20000).solve()
    _kkt_checks(prob, out, eps)
    meta = prob["meta"]
    nv = meta["nvar"]
    x = out["x"][:nv]
    xf = fista_lasso(meta["F"], meta["g"], meta["mu"], iters=30000)
    obj = lambda v: 0.5 * np.sum((meta["F"] @ v - meta["g"]) ** 2) + meta["mu"] * np.abs(v).sum()
    assert abs(obj(x) - obj(xf)) <= 1e-7 * (1 + abs(obj(xf)))
    np.testing.assert_allclose(x, xf, atol=1e-4)
    # LASSO subgradient condition F^T(g - F x) in mu d||x||_1
    gr = meta["F"].T @ (meta["g"] - meta["F"] @ x)
    assert np.all(np.abs(gr) <= meta["mu"] * (1 + 1e-4))
    # reported objective equals the LASSO objective at the optimum
    assert abs(out["info"].pobj - obj(x)) <= 1e-6 * (1 + abs(obj(x)))


@pytest.mark.parametrize("seed", [0, 1])
def test_planted_optimum(seed):
    prob = W.planted(seed=20 + seed, n=120, l=120, soc=[6] * 6 + [1, 2], psd=[3, 4], f=3, nnz=2500)
    eps = 1e-8
    out = O.Oracle(prob, direction=O.DIR_AA, mem=10, eps=eps, max_iters=20000).solve()
    _kkt_checks(prob, out, eps)
    pstar = prob["c"] @ prob["xstar"]
    assert abs(out["info"].pobj - pstar) <= 1e-6 * (1 + abs(pstar))
    assert abs(out["info"].dobj - pstar) <= 1e-6 * (1 + abs(pstar))


def test_infeasible_certificate():
    prob = W.infeasible(seed=3, n=80, l=80, nnz=1500)
    eps = 1e-7
    out = O.Oracle(prob, direction=O.DIR_AA, mem=10, eps=eps, max_iters=20000).solve()
    info = out["info"]
    assert info.status == O.INFEASIBLE, info
    y = out["y"]
    assert abs(prob["b"] @ y + 1) <= 1e-9
    assert np.linalg.norm(prob["A"].T @ y) * np.linalg.norm(prob["b"]) <= eps * 1.0001
    check_in_cone(prob, y, dual=True, tol=1e-9)
    assert np.all(np.isnan(out["x"]))


def test_unbounded_certificate():
    prob = W.unbounded(seed=4, n=80, l=80, nnz=1500)
    eps = 1e-7
    out = O.Oracle(prob, direction=O.DIR_AA, mem=10, eps=eps, max_iters=20000).solve()
    info = out["info"]
    assert info.status == O.UNBOUNDED, info
    x, s = out["x"], out["s"]
    assert abs(prob["c"] @ x + 1) <= 1e-9
    assert np.linalg.norm(prob["A"] @ x + s) * np.linalg.norm(prob["c"]) <= eps * 1.0001
    check_in_cone(prob, s, dual=False, tol=1e-9)


def test_warm_start_from_solution_terminates_immediately():
    prob = W.lasso(seed=2)
    o1 = O.Oracle(prob, eps=1e-8, max_iters=20000).solve()
    out = O.Oracle(prob, eps=1e-7, max_iters=20000, warm_u=o1["u"]).solve()
    assert out["info"].status == O.SOLVED and out["info"].iters <= 2


def test_planted_optimum_with_exponential_cones():
    # planted complementary pairs on primal and dual exponential cone blocks (all three cases),
    # mixed with orthant and SOC rows: the oracle must reach the planted objective
    prob = W.planted(seed=21, n=60, l=30, soc=[5, 4], ep=9, ed=6, nnz=900)
    eps = 1e-7
    out = O.Oracle(prob, eps=eps, max_iters=20000).solve()
    assert out["info"].status == O.SOLVED, out["info"]
    pstar = prob["c"] @ prob["xstar"]
    assert abs(out["info"].pobj - pstar) <= 10 * eps * (1 + abs(pstar))
    check_in_cone(prob, out["s"], dual=False, tol=1e-6)
    check_in_cone(prob, out["y"], dual=True, tol=1e-6)


@pytest.mark.parametrize("lam", [2.0, 8.0])
def test_logreg_vs_fista(lam):
    # the l1-regularised logistic regression of Sec. 5.4 in conic form (two exponential cones per
    # sample) against an independent proximal-gradient solve of the same objective
    from tests.helpers import fista_logreg
    prob = W.logreg(seed=3, p=20, q=30, lam=lam)
    out = O.Oracle(prob, eps=1e-9, max_iters=50000).solve()
    assert out["info"].status == O.SOLVED, out["info"]
    p = prob["meta"]["p"]
    w = out["x"][:p]
    wf, objf = fista_logreg(prob["meta"]["samples"], lam, iters=40000)
    obj = lam * np.abs(w).sum() + np.logaddexp(0.0, prob["meta"]["samples"] @ w).sum()
    assert abs(out["info"].pobj - objf) <= 1e-6 * (1 + abs(objf))
    assert abs(obj - objf) <= 1e-6 * (1 + abs(objf))
    np.testing.assert_allclose(w, wf, atol=1e-4)
