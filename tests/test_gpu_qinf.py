"""GPU parity for model CCM with q = inf (the max norm on x_i - x_j; Sec. 1 allows
any q >= 1): ccm_solve_path(q = CCM_Q_INF) against the q = inf CPU oracle — X
within 1e-6 relative of the oracle solved to KKT <= 1e-11, the q = inf KKT
residuals and gap recomputed by the oracle from the GPU's (X, U) <= 1e-6, labels
equal to the oracle's labelling of the GPU's X — on short rows and on long rows
(the ring kernels with the diag(mask) - s s^T Jacobian), in both precisions. The
device finds the l1-ball threshold by an active-set iteration and the oracle by
sorting, so agreement also checks one projection against the other."""
import math

import numpy as np
import pytest

from oracle import exact1d
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


def _dev(A, E, w):
    dev = torch.device("cuda:0")
    return (torch.tensor(A, device=dev), torch.tensor(E, dtype=torch.int32, device=dev),
            torch.tensor(w, device=dev))


_ORACLE = {}


def _check(ccm, key, A, E, w, gammas, precision):
    if key not in _ORACLE:          # both precisions compare with one oracle path
        _ORACLE[key] = ossnal.solve_path(A, E, w, gammas, tol=1e-11, q=np.inf)[0]
    Xo = _ORACLE[key]
    At, Et, wt = _dev(A, E, w)
    X, lab, U, st = ccm.solve_path(At, Et, wt, gammas, q=math.inf, tol=SOLVE_TOL,
                                   return_U=True, precision=precision)
    X, U, lab = X.cpu().numpy(), U.cpu().numpy(), lab.cpu().numpy()
    for t, g in enumerate(gammas):
        assert st[t]["status"] == 0, st[t]
        rel = np.linalg.norm(X[t] - Xo[t]) / max(np.linalg.norm(Xo[t]), 1e-300)
        assert rel <= TOL, (t, g, rel, st[t])
        res = okkt.kkt(A, E, w, g, X[t], U[t], q=np.inf)
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, g, res)
        assert abs(res["kkt"] - st[t]["kkt"]) <= 1e-8 + 1e-3 * res["kkt"], (res, st[t])
        assert res["dual_infeas"] <= 1e-12
        assert np.array_equal(lab[t], olabels.labels(X[t], E)), t


@pytest.mark.parametrize("precision", [1, 0])
def test_qinf_short_rows_match_oracle(ccm, precision):
    A, E, w = _problem(31, 60, 5, 5)
    _check(ccm, "short", A, E, w, np.array([0.0, 0.05, 0.4, 2.0, 20.0]), precision)


@pytest.mark.parametrize("precision", [1, 0])
def test_qinf_long_rows_match_oracle(ccm, precision):
    A, E, w = _problem(32, 36, 150, 4)
    _check(ccm, "long", A, E, w, np.array([0.1, 1.0, 6.0]), precision)


def test_qinf_two_points_by_hand(ccm):
    """w = 1, a1 - a2 = (4, 1): differences (2, 1), (0.5, 0.5), (0, 0) at gamma =
    1, 2, 3 (derived by hand: the larger coordinate shrinks alone by 2 gamma until
    both are equal, then both, fusion at 2 gamma = 5); gamma = 1 leaves a support
    of one element, where the Newton Jacobian P_l is zero."""
    a = np.array([[5.0, 1.0], [1.0, 0.0]])
    At, Et, wt = _dev(a, np.array([[0, 1]]), np.array([1.0]))
    gam = [1.0, 2.0, 3.0]
    X, _, _, _ = ccm.solve_path(At, Et, wt, gam, q="inf", tol=1e-10)
    X = X.cpu().numpy()
    mid = np.array([3.0, 0.5])
    for t, z in enumerate([(2.0, 1.0), (0.5, 0.5), (0.0, 0.0)]):
        z = np.array(z)
        want = np.stack([mid + z / 2, mid - z / 2])
        assert np.abs(X[t] - want).max() <= 1e-8, (gam[t], X[t], want)


def test_qinf_one_dimension_is_exact_1d_path_and_equals_q2(ccm):
    """d = 1: every q-norm is |.|, so q = inf, q = 2 and the certified exact 1-D
    path (complete graph, unit weights) coincide."""
    a = np.random.default_rng(33).normal(size=(14, 1))
    E = exact1d.complete_graph(14)
    At, Et, wt = _dev(a, E, np.ones(E.shape[0]))
    gam = [0.01, 0.05, 0.3]
    Xi, _, _, _ = ccm.solve_path(At, Et, wt, gam, q=ccm.Q_INF, tol=1e-10, engine=1)
    X2, _, _, _ = ccm.solve_path(At, Et, wt, gam, q=2, tol=1e-10, engine=1)
    Xi, X2 = Xi.cpu().numpy(), X2.cpu().numpy()
    for t, g in enumerate(gam):
        ex = exact1d.solve(a[:, 0], g)
        assert np.abs(Xi[t, :, 0] - ex).max() <= 1e-7, g
        assert np.abs(Xi[t] - X2[t]).max() <= 1e-7, g


def test_qinf_block_engine_rejected(ccm):
    A, E, w = _problem(34, 20, 3, 3)
    At, Et, wt = _dev(A, E, w)
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, Et, wt, [0.1], q="inf", engine=2)
