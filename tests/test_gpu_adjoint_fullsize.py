"""The adjoint workload at its full size: n = 20,000 points in d = 64 (20
Gaussian components N(0, 16 I), std 1), k = 10, phi = 1/median, 10 gammas
log-spaced in [1e-2, 10].

* Forward path, by properties that hold at any size (the oracle cannot solve
  this path in seconds): KKT residuals and relative gap (Sec. 4) recomputed by
  the oracle from the GPU's (X, U) <= 1e-6; mean preservation
  sum_i x_i = sum_i a_i; labels equal to the oracle's labelling rule applied to
  the GPU's X.
* dL/dA and dL/dw of L = sum_t ||X*(gamma_t) - T||_F^2 (implicit
  differentiation; not in the paper) against central differences of GPU path
  solves: step h = 1e-6 along 20 random directions of unit Frobenius norm in
  (A, w), solves at KKT <= 1e-11 in float64. Directions whose +-h solves
  change any label are skipped and counted; at least 10 must remain.
  L(+h) - L(-h) is formed as sum_t <X+ - X-, X+ + X- - 2T>, so the rounding of
  L itself (about 1e-16 L) does not enter the difference quotient.
"""
import numpy as np
import pytest

import synth
from oracle import kkt as okkt
from oracle import labels as olabels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, SOLVE_TOL = 1e-6, 2e-7


@pytest.fixture(scope="module")
def ccm():
    import paper_2501_15964_b300 as m
    return m


@pytest.fixture(scope="module")
def problem(ccm):
    A, _, wl = synth.make_workload("gmm20k_d64", 0)
    At = torch.tensor(A, device="cuda:0")
    Et, wt, _ = ccm.build_graph(At, wl.k, wl.phi)
    gam = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    return A, At, Et, wt, gam


def test_adjoint_workload_forward_full_size(ccm, problem):
    A, At, Et, wt, gam = problem
    E = Et.cpu().numpy().astype(np.int64)
    w = wt.cpu().numpy()
    X, L, U, st = ccm.solve_path(At, Et, wt, gam, tol=SOLVE_TOL, return_U=True)
    sA = A.sum(0)
    for t, g in enumerate(gam):
        Xt = X[t].cpu().numpy()
        assert st[t]["status"] == 0, st[t]
        res = okkt.kkt(A, E, w, g, Xt, U[t].cpu().numpy())
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, g, res)
        np.testing.assert_allclose(Xt.sum(0), sA, rtol=0, atol=1e-6 * (1 + np.abs(sA).max()))
        lab = L[t].cpu().numpy()
        assert np.array_equal(lab, olabels.labels(Xt, E))
        assert st[t]["n_clusters"] == lab.max() + 1
    # the path spans the fusion range
    assert st[-1]["n_clusters"] < st[0]["n_clusters"]


def test_adjoint_workload_central_differences(ccm, problem):
    A, At, Et, wt, gam = problem
    n, d = A.shape
    Tt = torch.tensor(synth.adjoint_target(0, n, d), device="cuda:0")
    kw = dict(tol=1e-11, precision=0)
    X, L, _, st = ccm.solve_path(At, Et, wt, gam, **kw)
    dA, dw = ccm.path_vjp(At, Et, wt, gam, X, 2.0 * (X - Tt))
    rng = np.random.default_rng(20)
    h = 1e-6
    kept, skipped, errs = 0, 0, []
    for _ in range(20):
        VA = rng.standard_normal(A.shape)
        Vw = rng.standard_normal(wt.shape[0])
        nrm = np.sqrt(np.sum(VA ** 2) + np.sum(Vw ** 2))
        VA = torch.tensor(VA / nrm, device="cuda:0")
        Vw = torch.tensor(Vw / nrm, device="cuda:0")
        Xp, Lp, _, _ = ccm.solve_path(At + h * VA, Et, wt + h * Vw, gam, **kw)
        Xm, Lm, _, _ = ccm.solve_path(At - h * VA, Et, wt - h * Vw, gam, **kw)
        if not (torch.equal(Lp, L) and torch.equal(Lm, L)):
            skipped += 1
            continue
        fd = float(torch.sum((Xp - Xm) * (Xp + Xm - 2.0 * Tt))) / (2 * h)
        an = float(torch.sum(dA * VA) + torch.sum(dw * Vw))
        errs.append(abs(fd - an) / (1 + abs(an)))
        kept += 1
    assert kept >= 10, (kept, skipped)
    assert max(errs) <= 1e-4, (max(errs), errs)
