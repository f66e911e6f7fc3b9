"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle.

Single operators of Eq. (drs) are compared element by element:
  Pi_C            identical arithmetic up to rounding      -> 1e-12 relative
  (I+Q)^{-1}      both CG to 1e-14 relative residual       -> 1e-9 relative
  T, R            composition of the two                   -> 1e-9 relative
Whole solves are iterations whose paths diverge with rounding, so parity is
judged on what is unique: the status, the GPU's own KKT residuals (<= eps,
recomputed here in FP64 from the returned x, y, s), the objective within
10 eps (1 + |p*|), and x itself where the solution is unique.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06477_gb300 import binding as B
from paper_1903_06477_gb300 import workloads as W
from tests.helpers import check_in_cone

pytestmark = pytest.mark.gpu


def _problems():
    return {
        "lasso": W.lasso(seed=0),
        "planted_mixed_cones": W.planted(seed=2, n=70, l=50, soc=[1, 2, 3, 7, 40], psd=[1, 2, 3, 5], f=3, nnz=1500),
        "portfolio": W.portfolio(seed=3, k=60),
        "planted_c2_small": W.c2_planted(seed=1, scale=0.01),
        "planted_exp_cones": W.planted(seed=21, n=60, l=30, soc=[5, 4], ep=9, ed=6, nnz=900),
        "logreg": W.logreg(seed=3, p=20, q=30, lam=2.0),
    }


PROBS = _problems()
TEAMS = [B.TEAM_BLOCK, B.TEAM_GRID]


def _kkt(prob, x, y, s):
    A, b, c = prob["A"], prob["b"], prob["c"]
    pr = np.linalg.norm(A @ x + s - b) / (1 + np.linalg.norm(b))
    dr = np.linalg.norm(A.T @ y + c) / (1 + np.linalg.norm(c))
    cx, by = c @ x, b @ y
    gap = abs(cx + by) / (1 + abs(cx) + abs(by))
    return pr, dr, gap


@pytest.mark.parametrize("team", TEAMS)
@pytest.mark.parametrize("name", list(PROBS))
def test_project_cone_parity(name, team):
    prob = PROBS[name]
    work = B.Work(prob, team=team, cg_rtol=1e-14)
    orc = O.Oracle(prob, cg_rtol=1e-14)
    rng = np.random.default_rng(0)
    for scale in (0.1, 1.0, 30.0):
        v = rng.standard_normal(work.N) * scale
        v[-1] = -abs(v[-1]) if scale == 1.0 else v[-1]
        out = work.project_cone(v)
        ref = orc.proj_C(v)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * (1 + np.abs(ref).max()))


@pytest.mark.parametrize("team", TEAMS)
@pytest.mark.parametrize("name", list(PROBS))
def test_linsys_and_T_parity(name, team):
    prob = PROBS[name]
    work = B.Work(prob, team=team, cg_rtol=1e-14, cg_max=5000)
    orc = O.Oracle(prob, cg_rtol=1e-14, cg_max=5000)
    rng = np.random.default_rng(1)
    for slot in (0, 1, 0):
        r = rng.standard_normal(work.N) * 3
        out = work.linsys(r, slot=slot)
        ref = orc.linsys(r, slot=slot)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9 * (1 + np.abs(ref).max()))
    u = rng.standard_normal(work.N)
    Tu, Ru = work.apply_T(u)
    Tr, Rr = orc.apply_T(u)
    np.testing.assert_allclose(Tu, Tr, rtol=0, atol=1e-9 * (1 + np.abs(Tr).max()))
    np.testing.assert_allclose(Ru, Rr, rtol=0, atol=1e-9 * (1 + np.abs(Tr).max()))


@pytest.mark.parametrize("team", TEAMS)
@pytest.mark.parametrize("direction", [B.DIR_AA, B.DIR_RB, B.DIR_AA_QR])
@pytest.mark.parametrize("name", list(PROBS))
def test_solve_parity_fp64(name, direction, team):
    prob = PROBS[name]
    eps = 1e-6
    c0 = 0.1 if direction == B.DIR_RB else 0.99
    kw = dict(direction=direction, mem=10, c0=c0, eps=eps, max_iters=20000, cg_rtol=1e-12)
    work = B.Work(prob, team=team, **kw)
    x, y, s, info = work.solve()
    okw = dict(kw)
    okw["cg_rtol"] = 1e-12
    ref = O.Oracle(prob, **okw).solve()
    assert info["status"] == B.SOLVED == ref["info"].status, (info, ref["info"])
    assert max(info["pr"], info["dr"], info["gap"]) <= eps
    pr, dr, gap = _kkt(prob, x, y, s)
    assert max(pr, dr, gap) <= eps * 1.01, (pr, dr, gap)
    check_in_cone(prob, s, dual=False, tol=1e-7 * (1 + np.abs(s).max()))
    check_in_cone(prob, y, dual=True, tol=1e-7 * (1 + np.abs(y).max()))
    p_ref = ref["info"].pobj
    assert abs(info["pobj"] - p_ref) <= 10 * eps * (1 + abs(p_ref))
    if "xstar" in prob:
        pstar = prob["c"] @ prob["xstar"]
        assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))
    if name == "lasso":
        nv = prob["meta"]["nvar"]
        np.testing.assert_allclose(x[:nv], ref["x"][:nv], atol=5e-4)


def test_km_iterates_match_oracle():
    """d = 0 and K0 off: both sides run the KM iteration (Eq. km); the iterates
    agree to CG accuracy after a fixed number of steps."""
    prob = PROBS["planted_mixed_cones"]
    kw = dict(direction=B.DIR_NONE, c0=0.0, eps=1e-30, max_iters=30, cg_rtol=1e-14, cg_max=5000)
    for team in TEAMS:
        work = B.Work(prob, team=team, **kw)
        work.solve()
        u = work.get_u()
        okw = dict(kw)
        okw["direction"] = O.DIR_NONE
        ref = O.Oracle(prob, **okw).solve()
        np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-8 * (1 + np.abs(ref["u"]).max()))


@pytest.mark.parametrize("branch", ["K0", "K1"])
@pytest.mark.parametrize("direction,mem", [(B.DIR_AA, 3), (B.DIR_RB, 2), (B.DIR_AA_QR, 3), (B.DIR_AA_QR, 5)])
def test_k0_k1_iterates_match_oracle(direction, mem, branch):
    """Every step forced to K0 (c0 = 1e300) or to K1 at alpha = 1 (c0 = 0,
    c1 = 1e300): u+ = u + d with Anderson or restarted Broyden directions (on
    the oracle side that path is pinned step by step against textbook
    Anderson acceleration and a dense Broyden iteration); after a dozen steps
    the GPU's iterate equals the oracle's to CG accuracy."""
    prob = PROBS["planted_mixed_cones"]
    iters = 12
    forced = dict(c0=1e300) if branch == "K0" else dict(c0=0.0, c1=1e300)
    kw = dict(direction=direction, mem=mem, eps=1e-30, max_iters=iters, cg_rtol=1e-14, cg_max=5000, **forced)
    okw = dict(kw, direction={B.DIR_AA: O.DIR_AA, B.DIR_RB: O.DIR_RB, B.DIR_AA_QR: O.DIR_AA_QR}[direction])
    ref = O.Oracle(prob, **okw).solve()
    key = "k0" if branch == "K0" else "k1"
    assert getattr(ref["info"], key) == iters
    for team in TEAMS:
        work = B.Work(prob, team=team, **kw)
        _, _, _, info = work.solve()
        assert info[key] == iters and info["backtracks"] == 0, info
        u = work.get_u()
        np.testing.assert_allclose(u, ref["u"], rtol=0, atol=1e-8 * (1 + np.abs(ref["u"]).max()))


@pytest.mark.parametrize("team", TEAMS)
def test_infeasible_and_unbounded(team):
    eps = 1e-7
    for kind, prob in (("inf", W.infeasible(seed=3, n=80, l=80, nnz=1500)),
                       ("unb", W.unbounded(seed=4, n=80, l=80, nnz=1500))):
        work = B.Work(prob, team=team, eps=eps, max_iters=20000, cg_rtol=1e-12)
        x, y, s, info = work.solve()
        if kind == "inf":
            assert info["status"] == B.INFEASIBLE, info
            assert abs(prob["b"] @ y + 1) <= 1e-8
            assert np.linalg.norm(prob["A"].T @ y) * np.linalg.norm(prob["b"]) <= eps * 1.01
            check_in_cone(prob, y, dual=True, tol=1e-9)
            assert np.all(np.isnan(x))
        else:
            assert info["status"] == B.UNBOUNDED, info
            assert abs(prob["c"] @ x + 1) <= 1e-8
            assert np.linalg.norm(prob["A"] @ x + s) * np.linalg.norm(prob["c"]) <= eps * 1.01
            check_in_cone(prob, s, dual=False, tol=1e-9)


@pytest.mark.parametrize("team", TEAMS)
@pytest.mark.parametrize("name", list(PROBS))
def test_refined_linsys_matches_oracle(name, team):
    """(I+Q)^{-1} by iterative refinement (FP64 residuals, FP32 CG corrections
    with the FP32 copy of A) reaches the same FP64 solution as plain CG."""
    prob = PROBS[name]
    work = B.Work(prob, team=team, precision=B.MIXED, cg_rtol=1e-14, cg_max=5000)
    orc = O.Oracle(prob, cg_rtol=1e-14, cg_max=5000)
    rng = np.random.default_rng(11)
    for slot in (0, 1, 0):
        r = rng.standard_normal(work.N) * 3
        out = work.linsys(r, slot=slot + 2)
        ref = orc.linsys(r, slot=slot)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9 * (1 + np.abs(ref).max()))


@pytest.mark.parametrize("precision", [B.FP64, B.MIXED])
@pytest.mark.parametrize("name", list(PROBS))
def test_direct_linsys_matches_oracle(name, precision):
    """(I+Q)^{-1} with I + A^T A factored L L^T at setup (one CTA per instance)
    against the oracle's CG to 1e-14; then whole solves with direct linear
    systems (both phases factored in their own precision) reach eps."""
    prob = PROBS[name]
    work = B.Work(prob, team=B.TEAM_BLOCK, linsys_direct=1, precision=precision, cg_rtol=1e-14, cg_max=5000)
    orc = O.Oracle(prob, cg_rtol=1e-14, cg_max=5000)
    rng = np.random.default_rng(12)
    for slot in (0, 1, 0):
        r = rng.standard_normal(work.N) * 3
        out = work.linsys(r, slot=slot)
        ref = orc.linsys(r, slot=slot)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9 * (1 + np.abs(ref).max()))
    eps = 1e-6
    w2 = B.Work(prob, team=B.TEAM_BLOCK, linsys_direct=1, precision=precision, eps=eps, max_iters=20000)
    x, y, s, info = w2.solve()
    ref = O.Oracle(prob, eps=eps, max_iters=20000).solve()
    assert info["status"] == B.SOLVED == ref["info"].status, info
    assert max(_kkt(prob, x, y, s)) <= 1.01 * eps
    assert abs(info["pobj"] - ref["info"].pobj) <= 10 * eps * (1 + abs(ref["info"].pobj))


@pytest.mark.parametrize("team", TEAMS)
@pytest.mark.parametrize("resume,refine", [(1, 1), (0, 0), (1, 0), (0, 1)])
def test_mixed_handover_modes(team, resume, refine):
    """Every combination of the FP32 -> FP64 hand-over (resume the loop state
    or restart) and of the FP64 phase's linear solves (refinement or plain
    FP64 CG) ends at the FP64 tolerance with the planted objective."""
    prob = W.c2_planted(seed=2, scale=0.02)
    eps = 1e-6
    work = B.Work(prob, team=team, precision=B.MIXED, eps=eps, max_iters=20000, cg_adapt=1e-2,
                  mixed_switch=1e-5, mixed_resume=resume, mixed_refine=refine)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    pr, dr, gap = _kkt(prob, x, y, s)
    assert max(pr, dr, gap) <= eps * 1.01
    pstar = prob["c"] @ prob["xstar"]
    assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))
    if refine and info["iters"] > info["iters_fp32"]:
        assert info["ir_sweeps"] > 0 and info["mat_passes_ir"] > 0, info
    if not refine:
        assert info["ir_sweeps"] == 0 and info["mat_passes_ir"] == 0, info


@pytest.mark.parametrize("team", TEAMS)
def test_mixed_precision_reaches_fp64_tolerance(team):
    prob = W.c2_planted(seed=2, scale=0.02)
    eps = 1e-6
    work = B.Work(prob, team=team, precision=B.MIXED, eps=eps, max_iters=20000)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    assert info["iters_fp32"] > 0
    pr, dr, gap = _kkt(prob, x, y, s)
    assert max(pr, dr, gap) <= eps * 1.01
    pstar = prob["c"] @ prob["xstar"]
    assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))


@pytest.mark.parametrize("team", TEAMS)
def test_exp_cone_projection_extreme_points(team):
    """Pi_C on exponential-cone rows at points that exercise every branch of the
    projection: inside K, in the polar cone, the face case, roots far beyond
    the scan range (|rho| in the hundreds), and magnitudes from 1e-6 to 1e6."""
    prob = W.planted(seed=4, n=20, l=4, ep=40, ed=40, nnz=300)
    work = B.Work(prob, team=team)
    orc = O.Oracle(prob)
    rng = np.random.default_rng(7)
    n, m = work.n, work.m
    for trial in range(6):
        v = rng.standard_normal(work.N)
        e = v[n + 4:n + m].reshape(-1, 3)
        if trial == 1:
            e[:, 2] = np.abs(e[:, 2]) * 1e-4   # x3 tiny positive, x2 negative: roots near 1 - x2/x3
            e[:, 1] = -np.abs(e[:, 1])
        if trial == 2:
            e *= np.exp(rng.uniform(-14, 14, (len(e), 1)))
        if trial == 3:
            e[:, 1] = np.abs(e[:, 1]) * 1e-5  # x2 tiny positive
        v[n + 4:n + m] = e.ravel()
        out = work.project_cone(v)
        ref = orc.proj_C(v)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * (1 + np.abs(ref).max()))


def test_edge_cases():
    # zero-cone only rows, dimension-1 SOCs, an empty row, PSD of order 1
    rng = np.random.default_rng(9)
    prob = W.planted(seed=9, n=15, l=4, soc=[1, 1, 2], psd=[1], f=3, nnz=60)
    A = prob["A"].tolil()
    A[4, :] = 0  # an empty orthant row: s_4 = b_4
    A = A.tocsr()
    A.eliminate_zeros()
    prob = dict(prob, A=A, b=A @ prob["xstar"] + prob["sstar"])
    ycheck = prob["ystar"].copy()
    prob["c"] = -(A.T @ ycheck)
    for team in TEAMS:
        work = B.Work(prob, team=team, eps=1e-7, max_iters=50000, cg_rtol=1e-12)
        x, y, s, info = work.solve()
        assert info["status"] == B.SOLVED, info
        pr, dr, gap = _kkt(prob, x, y, s)
        assert max(pr, dr, gap) <= 1.01e-7
        v = rng.standard_normal(work.N)
        np.testing.assert_allclose(work.project_cone(v), O.Oracle(prob).proj_C(v), atol=1e-12)


def test_invalid_inputs_rejected():
    prob = W.lasso(seed=0)
    bad = dict(prob)
    bad["b"] = prob["b"].copy()
    bad["b"][3] = np.nan
    with pytest.raises(B.SCSError):
        B.Work(bad)
    bad = dict(prob, l=prob["l"] + 1)
    with pytest.raises(B.SCSError):
        B.Work(bad)
    with pytest.raises(B.SCSError):
        B.Work(prob, mem=99)


@pytest.mark.parametrize("direct", [0, 1])
@pytest.mark.parametrize("precision", [B.FP64, B.MIXED])
def test_batch_parity(precision, direct):
    probs = [W.portfolio(seed=100 + i, k=int(k)) for i, k in enumerate(np.linspace(20, 140, 24))]
    eps = 1e-6
    batch = B.Batch(probs, precision=precision, eps=eps, max_iters=20000, cg_rtol=1e-12, linsys_direct=direct)
    xs, ys, ss, infos = batch.solve()
    for p, x, y, s, info in zip(probs, xs, ys, ss, infos):
        assert info["status"] == B.SOLVED, info
        pr, dr, gap = _kkt(p, x, y, s)
        assert max(pr, dr, gap) <= eps * 1.01
        ref = O.Oracle(p, eps=eps, max_iters=20000).solve()
        assert abs(info["pobj"] - ref["info"].pobj) <= 10 * eps * (1 + abs(ref["info"].pobj))


def test_device_pointers_roundtrip():
    torch = pytest.importorskip("torch")
    prob = PROBS["lasso"]
    work = B.Work(prob, eps=1e-6)
    xd = torch.empty(work.n, dtype=torch.float64, device="cuda")
    yd = torch.empty(work.m, dtype=torch.float64, device="cuda")
    sd = torch.empty(work.m, dtype=torch.float64, device="cuda")
    _, _, _, info = work.solve(xd, yd, sd)
    x2, y2, s2, info2 = work.solve()
    assert info["status"] == info2["status"] == B.SOLVED
    np.testing.assert_array_equal(xd.cpu().numpy(), x2)
    np.testing.assert_array_equal(sd.cpu().numpy(), s2)


def test_repeat_solves_are_deterministic():
    prob = PROBS["planted_c2_small"]
    work = B.Work(prob, team=B.TEAM_GRID, eps=1e-6)
    a = work.solve()
    b = work.solve()
    np.testing.assert_array_equal(a[0], b[0])
    assert a[3]["iters"] == b[3]["iters"]


@pytest.mark.parametrize("team", TEAMS)
def test_residuals_entry_matches_numpy(team):
    """scs_residuals evaluates Sec. 4.3's pr, dr, gap for any candidate."""
    prob = PROBS["planted_mixed_cones"]
    work = B.Work(prob, team=team, eps=1e-6, max_iters=20000)
    x, y, s, info = work.solve()
    out = work.residuals(x, y, s)
    ref = _kkt(prob, x, y, s)
    np.testing.assert_allclose(out, ref, rtol=1e-9, atol=1e-15)
    rng = np.random.default_rng(4)
    xr, yr, sr = rng.standard_normal(work.n), rng.standard_normal(work.m), rng.standard_normal(work.m)
    np.testing.assert_allclose(work.residuals(xr, yr, sr), _kkt(prob, xr, yr, sr), rtol=1e-12)


@pytest.mark.parametrize("team", TEAMS)
def test_psd_projection_large_blocks(team):
    """PSD blocks up to the largest supported order (64), odd orders padded."""
    prob = W.planted(seed=41, n=40, l=10, psd=[64, 33, 17, 2], nnz=2000)
    work = B.Work(prob, team=team)
    orc = O.Oracle(prob)
    rng = np.random.default_rng(7)
    for _ in range(2):
        v = rng.standard_normal(work.N) * 2
        np.testing.assert_allclose(work.project_cone(v), orc.proj_C(v), rtol=0, atol=1e-10)


def _psd_segments(prob, n):
    """(start, length) of each PSD block's svec rows in an HSDE vector (x, y, tau)."""
    o = n + prob["f"] + prob["l"] + int(sum(prob["q"]))
    segs = []
    for d in prob["s"]:
        segs.append((o, d * (d + 1) // 2))
        o += d * (d + 1) // 2
    return segs


@pytest.mark.parametrize("team", TEAMS)
def test_psd_fp32_recheck_redoes_blocks_in_fp64(team):
    """Sec. 2, cone (ii): the FP32 phase's eigensolves are checked in FP64 and a block above
    psd_recheck_tol is decomposed again in FP64.  With the bound 0 every block is redone: its
    projection is then the exact one of the FP32-rounded block, so (projection being
    1-Lipschitz) it lies within a few FP32 roundings of the FP64 oracle's, ||.||_F per block.
    With the default bound no converged FP32 eigensolve is redone."""
    prob = W.planted(seed=43, n=40, l=10, psd=[64, 33, 17, 2], nnz=2000)
    orc = O.Oracle(prob)
    u32 = 2.0 ** -24
    rng = np.random.default_rng(8)
    v = rng.standard_normal(40 + prob["A"].shape[0] + 1) * 2
    ref = orc.proj_C(v)
    segs = _psd_segments(prob, 40)
    forced = B.Work(prob, team=team, precision=B.MIXED, psd_recheck_tol=0.0)
    out, stats = forced.project_cone_prec(v, B.MIXED)
    assert stats[1] == len(prob["s"])
    for o, k in segs:
        err = np.linalg.norm(out[o:o + k] - ref[o:o + k])
        assert err <= 6 * u32 * np.linalg.norm(v[o:o + k]), (o, k, err)
    default = B.Work(prob, team=team, precision=B.MIXED)
    out_d, stats_d = default.project_cone_prec(v, B.MIXED)
    assert stats_d[1] == 0 and 0 < stats_d[0] < 1e-4
    for o, k in segs:
        assert np.linalg.norm(out_d[o:o + k] - ref[o:o + k]) <= 1e-4 * np.linalg.norm(v[o:o + k])
    # the FP64 form reports nothing and matches the oracle
    out64, stats64 = default.project_cone_prec(v, B.FP64)
    assert list(stats64) == [0.0, 0.0]
    np.testing.assert_allclose(out64, ref, rtol=0, atol=1e-10)


def test_psd_fp32_redo_in_a_solve():
    """A mixed solve with every FP32 PSD projection redone in FP64 still reaches eps."""
    prob = W.planted(seed=42, n=300, l=200, psd=[16] * 6 + [9, 33], nnz=6000)
    eps = 1e-5
    work = B.Work(prob, precision=B.MIXED, eps=eps, max_iters=20000, cg_adapt=1e-2, psd_recheck_tol=0.0)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    assert max(_kkt(prob, x, y, s)) <= eps * 1.01
    assert info["psd_redo_fp32"] >= info["iters_fp32"] * len(prob["s"])


@pytest.mark.parametrize("team", TEAMS)
def test_psd_projection_blocks_above_64(team):
    """PSD blocks above order 64 are decomposed in a global-memory workspace: Pi_C matches
    the oracle in FP64 (1e-10) and, as the FP32 phase runs it, within the FP32 bound with
    every block redone in FP64 (psd_recheck_tol = 0) and within 1e-4 ||X||_F by default."""
    prob = W.planted(seed=44, n=40, l=10, psd=[65, 100, 151, 7], nnz=3000)
    orc = O.Oracle(prob)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(40 + prob["A"].shape[0] + 1) * 2
    ref = orc.proj_C(v)
    work = B.Work(prob, team=team, precision=B.MIXED)
    np.testing.assert_allclose(work.project_cone(v), ref, rtol=0, atol=1e-10)
    out, stats = work.project_cone_prec(v, B.MIXED)
    assert 0 < stats[0] < 1e-4
    segs = _psd_segments(prob, 40)
    for o, k in segs:
        assert np.linalg.norm(out[o:o + k] - ref[o:o + k]) <= 1e-4 * np.linalg.norm(v[o:o + k])
    forced = B.Work(prob, team=team, precision=B.MIXED, psd_recheck_tol=0.0)
    out, stats = forced.project_cone_prec(v, B.MIXED)
    assert stats[1] == len(prob["s"])
    for o, k in segs:
        assert np.linalg.norm(out[o:o + k] - ref[o:o + k]) <= 6 * 2.0 ** -24 * np.linalg.norm(v[o:o + k])


@pytest.mark.parametrize("precision", [B.FP64, B.MIXED])
def test_sparse_pca_above_64_matches_oracle(precision):
    """The sparse-PCA SDP of Sec. 5.2 at d = 80 (one PSD block above 64): solved to eps, the
    objective within 10 eps (1 + |p*|) of the FP64 oracle's solve, Z in the PSD cone."""
    prob = W.pca_sdp(0, 80, 2.0)
    eps = 1e-5
    kw = dict(direction=B.DIR_AA, mem=10, eps=eps, max_iters=20000)
    work = B.Work(prob, precision=precision, cg_adapt=1e-2, **kw)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    assert max(_kkt(prob, x, y, s)) <= eps * 1.01
    check_in_cone(prob, s, dual=False, tol=1e-6)
    ref = O.Oracle(prob, **kw).solve()
    assert ref["info"].status == O.SOLVED
    pstar = ref["info"].pobj
    assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))


@pytest.mark.parametrize("precision", [B.FP64, B.MIXED])
def test_planted_sdp_small(precision):
    prob = W.planted(seed=42, n=300, l=200, psd=[16] * 6 + [9, 33], nnz=6000)
    eps = 1e-5
    work = B.Work(prob, precision=precision, eps=eps, max_iters=20000, cg_adapt=1e-2)
    x, y, s, info = work.solve()
    assert info["status"] == B.SOLVED, info
    pr, dr, gap = _kkt(prob, x, y, s)
    assert max(pr, dr, gap) <= eps * 1.01
    check_in_cone(prob, s, dual=False, tol=1e-6)
    check_in_cone(prob, y, dual=True, tol=1e-6)
    pstar = prob["c"] @ prob["xstar"]
    assert abs(info["pobj"] - pstar) <= 10 * eps * (1 + abs(pstar))
    if precision == B.MIXED:
        assert 0 < info["psd_resid_fp32"] < 1e-4  # FP64 recheck of the FP32 eigensolves
        assert info["psd_redo_fp32"] == 0  # converged FP32 eigensolves stay below the default bound


def test_batch_autotuned_mixed():
    probs = [W.portfolio(seed=500 + i, k=int(k)) for i, k in enumerate(np.linspace(20, 160, 96))]
    eps = 1e-5
    batch = B.Batch(probs, precision=B.MIXED, eps=eps, max_iters=20000, cg_adapt=1e-2)
    xs, ys, ss, infos = batch.solve()
    assert infos[0]["threads_per_block"] in (128, 256, 512, 1024)
    for p, x, y, s, info in zip(probs, xs, ys, ss, infos):
        assert info["status"] == B.SOLVED, info
        assert max(_kkt(p, x, y, s)) <= eps * 1.01
    # a second solve of the same batch gives the same answers
    xs2, _, _, infos2 = batch.solve()
    for a, b2 in zip(xs, xs2):
        np.testing.assert_array_equal(a, b2)
