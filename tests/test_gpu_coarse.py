"""Two-level preconditioner of the Newton-CG (options.coarse, grid engine, q = 2).

The coarse correction changes only the preconditioner of the CG that solves the
Newton system (Sec. 1: SSNAL), so the path must reach the same solution: X within
1e-6 relative of the Jacobi-only solve, and the oracle's KKT residuals and
relative gap (Sec. 4) of the returned (X, U) at most 1e-6. The correction must
actually engage on a path that fuses, and it must take fewer CG iterations.
"""
import numpy as np
import pytest

import synth
from oracle import kkt as okkt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6
SOLVE_TOL = 2e-7


@pytest.fixture(scope="module")
def ccm():
    import paper_2501_15964_b300 as m
    assert torch.cuda.is_available()
    return m


def _clustered(seed, n, d, n_comp, spread):
    rng = np.random.default_rng(seed)
    cent = rng.normal(0, spread, size=(n_comp, d))
    return cent[rng.integers(0, n_comp, n)] + rng.normal(size=(n, d))


@pytest.mark.parametrize("precision", [0, 1])
def test_coarse_correction_same_path_fewer_cg(ccm, precision):
    A = _clustered(23, 4000, 16, 8, 6.0)
    At = torch.tensor(A, device="cuda:0")
    Et, wt, _ = ccm.build_graph(At, 10, 0.0)
    E = Et.cpu().numpy().astype(np.int64)
    w = wt.cpu().numpy()
    g = synth.gamma_grid(1e-3, 10.0, 12)
    runs = {}
    for co in (0, 1):
        X, _, U, st = ccm.solve_path(At, Et, wt, g, tol=SOLVE_TOL, return_U=True,
                                     precision=precision, engine=1, coarse=co, profile=1)
        prof = ccm.last_profile()
        assert all(s["status"] == 0 for s in st), st
        runs[co] = (X.cpu().numpy(), U.cpu().numpy(), st, prof)
    X0, _, st0, p0 = runs[0]
    X1, U1, st1, p1 = runs[1]
    assert p0["coarse_steps"] == 0
    assert p1["coarse_steps"] > 0, p1
    assert 1 <= p1["coarse_max_aggregates"] <= 224, p1
    for t, gm in enumerate(g):
        assert np.linalg.norm(X1[t] - X0[t]) <= TOL * np.linalg.norm(X0[t]), t
        res = okkt.kkt(A, E, w, gm, X1[t], U1[t])
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, res)
    cg0 = sum(s["cg"] for s in st0)
    cg1 = sum(s["cg"] for s in st1)
    assert cg1 < cg0, (cg0, cg1)


def test_coarse_correction_long_rows_ring_operator(ccm):
    """d = 784 rows take the shared-memory ring operator; the coarse correction
    feeds it U = M^-1 R with unit Jacobi scalars."""
    A = _clustered(5, 1500, 784, 6, 1.5)
    At = torch.tensor(A, device="cuda:0")
    Et, wt, _ = ccm.build_graph(At, 10, 0.0)
    E = Et.cpu().numpy().astype(np.int64)
    w = wt.cpu().numpy()
    g = synth.gamma_grid(1e-2, 10.0, 8)
    X, _, U, st = ccm.solve_path(At, Et, wt, g, tol=SOLVE_TOL, return_U=True, engine=1,
                                 coarse=1, profile=1)
    prof = ccm.last_profile()
    assert all(s["status"] == 0 for s in st), st
    assert prof["coarse_steps"] > 0, prof
    X = X.cpu().numpy()
    U = U.cpu().numpy()
    for t, gm in enumerate(g):
        res = okkt.kkt(A, E, w, gm, X[t], U[t])
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, res)
