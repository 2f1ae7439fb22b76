"""GPU parity of the block engine and ccm_solve_path_batched against the CPU
oracle (model CCM, Sec. 1; gap of Sec. 4): many independent problems of
uneven size in one persistent launch."""
import numpy as np
import pytest

import synth
from oracle import graph as ograph
from oracle import kkt as okkt
from oracle import labels as olabels
from oracle import ssnal as ossnal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, SOLVE_TOL = 1e-6, 2e-7


@pytest.fixture(scope="module")
def ccm():
    import paper_2501_15964_b300 as m
    return m


def _problems(count, seed, n_lo=40, n_hi=160, d=16):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        K = int(rng.integers(2, 6))
        k = int(rng.integers(3, 8))
        A, _ = synth.gaussian_mixture(rng, n, d, K, 5.0, 0.5, 1.5, "equal", "normal")
        E, w, _ = ograph.build_graph(A, k, 0.0)
        out.append((A, E, w))
    return out


def _dev(A, E, w):
    return dict(A=torch.tensor(A, device="cuda:0"),
                edges=torch.tensor(E, dtype=torch.int32, device="cuda:0"),
                w=torch.tensor(w, device="cuda:0"))


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_matches_oracle(ccm, precision):
    probs = _problems(12, 7)
    gammas = synth.gamma_grid(1e-3, 1e2, 8)
    Xs, Ls, stats = ccm.solve_path_batched([_dev(*p) for p in probs], gammas, tol=SOLVE_TOL,
                                          precision=precision)
    for (A, E, w), X, L, st in zip(probs, Xs, Ls, stats):
        Xo, _, _ = ossnal.solve_path(A, E, w, gammas, tol=1e-11)
        X = X.cpu().numpy()
        L = L.cpu().numpy()
        for t, g in enumerate(gammas):
            assert st[t]["status"] == 0, st[t]
            assert st[t]["kkt"] <= TOL and st[t]["gap"] <= TOL
            rel = np.linalg.norm(X[t] - Xo[t]) / np.linalg.norm(Xo[t])
            assert rel <= TOL, (t, rel)
            assert np.array_equal(L[t], olabels.labels(X[t], E))
            assert st[t]["n_clusters"] == L[t].max() + 1


def test_block_engine_single_problem_kkt(ccm):
    """ccm_solve_path with the block engine: KKT and gap recomputed by the oracle
    from the GPU's (X, U)."""
    A, _, wl = synth.make_workload("gmm200_d2", 2)
    E, w, _ = ograph.build_graph(A, wl.k, wl.phi)
    g = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    P = _dev(A, E, w)
    X, L, U, st = ccm.solve_path(P["A"], P["edges"], P["w"], g, tol=SOLVE_TOL, return_U=True,
                                 engine=2)
    X = X.cpu().numpy()
    U = U.cpu().numpy()
    for t in range(len(g)):
        res = okkt.kkt(A, E, w, g[t], X[t], U[t])
        assert res["kkt"] <= TOL and res["gap"] <= TOL, res
        assert np.array_equal(L[t].cpu().numpy(), olabels.labels(X[t], E))


def test_batched_equals_single_block_runs(ccm):
    """A batch gives the same X (bitwise) as solving each problem alone with the
    block engine: the work queue changes only where a problem runs."""
    probs = _problems(5, 11, 30, 90, d=8)
    g = [0.01, 0.3, 3.0]
    Xs, Ls, _ = ccm.solve_path_batched([_dev(*p) for p in probs], g, tol=SOLVE_TOL)
    for (A, E, w), Xb, Lb in zip(probs, Xs, Ls):
        P = _dev(A, E, w)
        X1, L1, _, _ = ccm.solve_path(P["A"], P["edges"], P["w"], g, tol=SOLVE_TOL, engine=2)
        assert torch.equal(Xb, X1) and torch.equal(Lb, L1)


def test_batched_rejects_bad_problem(ccm):
    probs = _problems(2, 3, 30, 40, d=4)
    bad = _dev(*probs[1])
    E = bad["edges"].clone()
    E[0, 1] = 10 ** 6
    bad["edges"] = E
    with pytest.raises(ccm.CCMError):
        ccm.solve_path_batched([_dev(*probs[0]), bad], [0.1])


def test_batched_config_sized_problems(ccm):
    """Eight problems of the batched workload itself (n ~ U{500..5000}, d = 16,
    2-20 components, k ~ U{5..15}, phi = 1/median, 25 gammas): the batched X
    within 1e-6 relative of ccm_solve_path on the grid engine, whose (X, U) the
    oracle checks for KKT and relative gap (Sec. 4) <= 1e-6; labels of both
    equal to the oracle's labelling rule applied to the batched X."""
    probs = synth.batched_problems(0, count=8)
    assert min(p["A"].shape[0] for p in probs) >= 500
    gam = probs[0]["gammas"]
    dev = []
    for p in probs:
        A = torch.tensor(p["A"], device="cuda:0")
        E, w, _ = ccm.build_graph(A, p["k"], p["phi"])
        dev.append(dict(A=A, edges=E, w=w))
    Xs, Ls, stats = ccm.solve_path_batched(dev, gam, tol=SOLVE_TOL)
    for p, P, Xb, Lb, st in zip(probs, dev, Xs, Ls, stats):
        Xg, Lg, Ug, stg = ccm.solve_path(P["A"], P["edges"], P["w"], gam, tol=SOLVE_TOL,
                                         return_U=True, engine=1)
        E = P["edges"].cpu().numpy().astype(np.int64)
        w = P["w"].cpu().numpy()
        for t, g in enumerate(gam):
            assert st[t]["status"] == 0 and stg[t]["status"] == 0, (st[t], stg[t])
            assert st[t]["kkt"] <= TOL and st[t]["gap"] <= TOL
            xg = Xg[t].cpu().numpy()
            res = okkt.kkt(p["A"], E, w, g, xg, Ug[t].cpu().numpy())
            assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, res)
            xb = Xb[t].cpu().numpy()
            assert np.linalg.norm(xb - xg) <= TOL * np.linalg.norm(xg), t
            lab = olabels.labels(xb, E)
            assert np.array_equal(Lb[t].cpu().numpy(), lab)


def test_batched_autotuned_shape_matches_default(ccm):
    """A batch of >= 8 problems measures the candidate group shapes (lanes x
    quads per row) on a sample and keeps the fastest; whichever it picks, the
    solutions agree with the default shape's within 1e-6 and every gamma meets
    the tolerance."""
    probs = _problems(12, 23, 60, 200, d=16)
    dev = [_dev(*p) for p in probs]
    g = synth.gamma_grid(1e-3, 1e2, 6)
    Xt, Lt, st = ccm.solve_path_batched(dev, g, tol=SOLVE_TOL, autotune=1)
    prof = ccm.last_profile()
    assert (prof["block_lanes"], prof["block_quads"]) in [(4, 1), (2, 2), (1, 4)], prof
    ctx2 = ccm.Context(0)
    X0, L0, st0 = ccm.solve_path_batched(dev, g, tol=SOLVE_TOL, autotune=0, ctx=ctx2)
    assert ccm.last_profile(ctx2)["block_lanes"] == 4
    for a, b, s1 in zip(Xt, X0, st):
        assert all(s["status"] == 0 and s["kkt"] <= TOL and s["gap"] <= TOL for s in s1)
        a, b = a.cpu().numpy(), b.cpu().numpy()
        for t in range(len(g)):
            assert np.linalg.norm(a[t] - b[t]) <= TOL * np.linalg.norm(b[t])
