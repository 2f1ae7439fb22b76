"""GPU parity for model CCM with q = 1 (the l1 norm on x_i - x_j; Sec. 1 allows
any q >= 1): ccm_solve_path(q = 1) against the q = 1 CPU oracle — X within 1e-6
relative of the oracle solved to KKT <= 1e-11, the q = 1 KKT residuals and gap
recomputed by the oracle from the GPU's (X, U) <= 1e-6, labels equal to the
oracle's labelling of the GPU's X — on short rows and on long rows (the ring
kernels with the diagonal-mask Jacobian), in both precisions."""
import numpy as np
import pytest

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


def _problem(seed, n, d, k):
    rng = np.random.default_rng(seed)
    cent = rng.normal(0, 2, size=(3, d))
    A = cent[rng.integers(0, 3, n)] + rng.normal(size=(n, d))
    E, w, _ = ograph.build_graph(A, k, 0.0)
    w[::9] = 0.0                                            # inert edges
    return A, E, w


def _check(ccm, A, E, w, gammas, precision):
    Xo, _, _ = ossnal.solve_path(A, E, w, gammas, tol=1e-11, q=1)
    dev = torch.device("cuda:0")
    At = torch.tensor(A, device=dev)
    Et = torch.tensor(E, dtype=torch.int32, device=dev)
    wt = torch.tensor(w, device=dev)
    X, lab, U, st = ccm.solve_path(At, Et, wt, gammas, q=1, tol=SOLVE_TOL, return_U=True,
                                   precision=precision)
    X, U, lab = X.cpu().numpy(), U.cpu().numpy(), lab.cpu().numpy()
    for t, g in enumerate(gammas):
        assert st[t]["status"] == 0, st[t]
        rel = np.linalg.norm(X[t] - Xo[t]) / max(np.linalg.norm(Xo[t]), 1e-300)
        assert rel <= TOL, (t, g, rel, st[t])
        res = okkt.kkt(A, E, w, g, X[t], U[t], q=1)
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, g, res)
        assert abs(res["kkt"] - st[t]["kkt"]) <= 1e-8 + 1e-3 * res["kkt"], (res, st[t])
        assert res["dual_infeas"] <= 1e-12
        assert np.array_equal(lab[t], olabels.labels(X[t], E)), t


@pytest.mark.parametrize("precision", [1, 0])
def test_q1_short_rows_match_oracle(ccm, precision):
    A, E, w = _problem(1, 60, 5, 5)
    _check(ccm, A, E, w, np.array([0.0, 0.05, 0.4, 2.0, 20.0]), precision)


@pytest.mark.parametrize("precision", [1, 0])
def test_q1_long_rows_match_oracle(ccm, precision):
    A, E, w = _problem(2, 36, 150, 4)
    _check(ccm, A, E, w, np.array([0.1, 1.0, 6.0]), precision)


def test_q1_two_points_closed_form(ccm):
    a = np.array([[1.0, 2.0, 0.5], [4.0, -2.0, 0.3]])
    At = torch.tensor(a, device="cuda:0")
    Et = torch.tensor([[0, 1]], dtype=torch.int32, device="cuda:0")
    wt = torch.tensor([0.8], dtype=torch.float64, device="cuda:0")
    gam = [0.05, 0.5, 1.0, 3.0]
    X, _, _, _ = ccm.solve_path(At, Et, wt, gam, q=1, tol=1e-10)
    X = X.cpu().numpy()
    for t, g in enumerate(gam):
        D = a[0] - a[1]
        delta = np.sign(D) * np.maximum(np.abs(D) - 2 * g * 0.8, 0.0)
        want = np.stack([a.mean(0) + 0.5 * delta, a.mean(0) - 0.5 * delta])
        assert np.abs(X[t] - want).max() <= 1e-8, (g, X[t], want)


def test_q1_block_engine_rejected(ccm):
    A, E, w = _problem(3, 20, 3, 3)
    At = torch.tensor(A, device="cuda:0")
    Et = torch.tensor(E, dtype=torch.int32, device="cuda:0")
    wt = torch.tensor(w, device="cuda:0")
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, Et, wt, [0.1], q=1, engine=2)
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, Et, wt, [0.1], q=3)
