"""GPU ADMM and fast AMA (ccm_solve_path_admm / ccm_solve_path_ama, the paper's
second and third solvers, Sec. 1) against the CPU oracle: the same bar as the
SSNAL path — X within 1e-6 relative of the
oracle solved to KKT <= 1e-11, the KKT residuals and relative gap recomputed by
the oracle from the GPU's (X, U) <= 1e-6, labels equal to the oracle's
labelling of the GPU's X — on short rows and on long rows (the ring kernels)."""
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
    assert torch.cuda.is_available()
    return m


def _check(ccm, A, E, w, gammas, precision, solver="admm"):
    Xo, _, _ = ossnal.solve_path(A, E, w, gammas, tol=1e-11)
    dev = torch.device("cuda:0")
    At = torch.tensor(A, device=dev)
    Et = torch.tensor(E, dtype=torch.int32, device=dev)
    wt = torch.tensor(w, device=dev)
    fn = ccm.solve_path_admm if solver == "admm" else ccm.solve_path_ama
    X, lab, U, st = fn(At, Et, wt, gammas, tol=SOLVE_TOL, return_U=True, precision=precision)
    X, U, lab = X.cpu().numpy(), U.cpu().numpy(), lab.cpu().numpy()
    for t, g in enumerate(gammas):
        assert st[t]["status"] == 0, st[t]
        rel = np.linalg.norm(X[t] - Xo[t]) / max(np.linalg.norm(Xo[t]), 1e-300)
        assert rel <= TOL, (t, g, rel, st[t])
        res = okkt.kkt(A, E, w, g, X[t], U[t])
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, g, res)
        assert np.array_equal(lab[t], olabels.labels(X[t], E)), t
    return st


@pytest.mark.parametrize("precision", [1, 0])
def test_admm_gmm200_matches_oracle(ccm, precision):
    A, _, wl = synth.make_workload("gmm200_d2", 0, n=120)
    E, w, _ = ograph.build_graph(A, wl.k, wl.phi)
    gammas = np.array([0.0, 0.05, 0.5, 3.0])
    st = _check(ccm, A, E, w, gammas, precision)
    assert st[0]["outer"] <= 10          # gamma = 0: X = A at the first check


@pytest.mark.parametrize("precision", [1, 0])
def test_admm_long_rows_matches_oracle(ccm, precision):
    rng = np.random.default_rng(5)
    cent = rng.normal(0, 2, size=(3, 150))
    A = cent[rng.integers(0, 3, 48)] + rng.normal(size=(48, 150))
    E, w, _ = ograph.build_graph(A, 5, 0.0)
    _check(ccm, A, E, w, np.array([1.0, 8.0]), precision)


def test_ama_gmm200_matches_oracle(ccm):
    A, _, wl = synth.make_workload("gmm200_d2", 0, n=120)
    E, w, _ = ograph.build_graph(A, wl.k, wl.phi)
    _check(ccm, A, E, w, np.array([0.0, 0.05, 0.5, 3.0]), 0, solver="ama")


def test_ama_long_rows_matches_oracle(ccm):
    rng = np.random.default_rng(5)
    cent = rng.normal(0, 2, size=(3, 150))
    A = cent[rng.integers(0, 3, 48)] + rng.normal(size=(48, 150))
    E, w, _ = ograph.build_graph(A, 5, 0.0)
    _check(ccm, A, E, w, np.array([1.0, 8.0]), 0, solver="ama")
