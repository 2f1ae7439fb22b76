"""Full-size parity on the large workloads, by properties that hold at any size
(the oracle cannot solve these paths in seconds):

* kNN graph: sampled rows against the oracle's exhaustive search, one by one;
* path: KKT residuals and relative gap (Sec. 4) recomputed by the oracle from
  the GPU's (X, U) <= 1e-6, mean preservation sum_i x_i = sum_i a_i, and labels
  equal to the oracle's labelling rule applied to the GPU's X.

The gamma values are a spread subset of each workload's grid (solved as one
warm-started path), so the returned multipliers stay a few GB.
"""
import numpy as np
import pytest

import synth
from oracle import graph as ograph
from oracle import kkt as okkt
from oracle import labels as olabels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, SOLVE_TOL = 1e-6, 2e-7


@pytest.fixture(scope="module")
def ccm():
    import paper_2501_15964_b300 as m
    return m


def _sampled_knn_check(A, E, k, rows):
    n = A.shape[0]
    adj = {}
    for a, b in E[np.isin(E[:, 0], rows) | np.isin(E[:, 1], rows)]:
        adj.setdefault(int(a), set()).add(int(b))
        adj.setdefault(int(b), set()).add(int(a))
    Nr = ograph.knn_rows(A, k, rows)
    for r, i in enumerate(rows):
        nb = adj.get(int(i), set())
        assert set(Nr[r].tolist()) <= nb
        extra = sorted(nb - set(Nr[r].tolist()))
        if extra:
            Ne = ograph.knn_rows(A, k, np.array(extra))
            for t in range(len(extra)):
                assert i in Ne[t]


def _path_properties(ccm, A, E, w, gammas):
    At = torch.tensor(A, device="cuda:0")
    Et = torch.tensor(E, dtype=torch.int32, device="cuda:0")
    wt = torch.tensor(w, device="cuda:0")
    X, L, U, st = ccm.solve_path(At, Et, wt, gammas, tol=SOLVE_TOL, return_U=True)
    sA = A.sum(0)
    for t, g in enumerate(gammas):
        Xt = X[t].cpu().numpy()
        Ut = U[t].cpu().numpy()
        assert st[t]["status"] == 0, st[t]
        res = okkt.kkt(A, E, w, g, Xt, Ut)
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, g, res)
        np.testing.assert_allclose(Xt.sum(0), sA, rtol=0, atol=1e-6 * (1 + np.abs(sA).max()))
        assert np.array_equal(L[t].cpu().numpy(), olabels.labels(Xt, E))
        del Ut


@pytest.mark.parametrize("name", ["gmm200k_d50", "gmm200k_d50_medphi"])
def test_large_gmm_full_size(ccm, name):
    A, _, wl = synth.make_workload(name, 0)
    At = torch.tensor(A, device="cuda:0")
    Et, wt, phi = ccm.build_graph(At, wl.k, wl.phi)
    info = ccm.last_graph_info()
    # tensor-core candidates, every row certified by the error bound (no exhaustive
    # float64 search needed at this size)
    assert info["candidates"] == "tensor" and info["rows_exhaustive"] == 0, info
    E = Et.cpu().numpy().astype(np.int64)
    w = wt.cpu().numpy()
    n = A.shape[0]
    assert n * wl.k / 2 <= E.shape[0] <= n * wl.k
    rng = np.random.default_rng(1)
    _sampled_knn_check(A, E, wl.k, rng.choice(n, 12, replace=False))
    gam = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)[::6]
    _path_properties(ccm, A, E, w, gam)


def test_mnist_shape_full_size_path(ccm):
    A, _, wl = synth.make_workload("mnist10k_d784", 0)
    At = torch.tensor(A, device="cuda:0")
    Et, wt, phi = ccm.build_graph(At, wl.k, wl.phi)
    gam = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)[::8]
    _path_properties(ccm, A, Et.cpu().numpy().astype(np.int64), wt.cpu().numpy(), gam)
