"""GPU parity of ccm_solve_path against the CPU oracle (model CCM, Sec. 1;
gap of Sec. 4).

Bar: X within 1e-6 relative (Frobenius, per gamma) of the oracle solved to
KKT <= 1e-11; KKT residuals and the relative gap recomputed by the oracle from
the GPU's (X, U) <= 1e-6; labels bit-exact with the oracle's labelling of the
GPU's X, and with the oracle's labels of its own X where no edge distance lies
in the ambiguous band [1e-8, 1e-4].
"""
import numpy as np
import pytest

import synth
from oracle import graph as ograph
from oracle import kkt as okkt
from oracle import labels as olabels
from oracle import ssnal as ossnal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6
SOLVE_TOL = 2e-7


@pytest.fixture(scope="module")
def ccm():
    import paper_2501_15964_b300 as m
    assert torch.cuda.is_available()
    return m


def _to_dev(A, edges, w):
    dev = torch.device("cuda:0")
    return (torch.tensor(A, device=dev), torch.tensor(edges, dtype=torch.int32, device=dev),
            torch.tensor(w, device=dev))


def _ambiguous(X, edges):
    d = np.sqrt(np.sum((X[edges[:, 0]] - X[edges[:, 1]]) ** 2, axis=1))
    return np.any((d > 1e-8) & (d < 1e-4))


def _check_path(ccm, A, edges, w, gammas, precision, xtol=TOL, engine=0):
    Xo, _, _ = ossnal.solve_path(A, edges, w, gammas, tol=1e-11)
    At, Et, wt = _to_dev(A, edges, w)
    # the solver stops at KKT <= 2e-7 (tighter than the 1e-6 bar) so that X is also
    # within 1e-6 of the oracle: KKT <= 1e-6 alone left 2e-6 on one gamma
    X, lab, U, stats = ccm.solve_path(At, Et, wt, gammas, tol=SOLVE_TOL, return_U=True,
                                      precision=precision, engine=engine)
    X = X.cpu().numpy()
    U = U.cpu().numpy()
    lab = lab.cpu().numpy()
    for t, g in enumerate(gammas):
        assert stats[t]["status"] == 0, stats[t]
        den = max(np.linalg.norm(Xo[t]), 1e-300)
        rel = np.linalg.norm(X[t] - Xo[t]) / den
        assert rel <= xtol, (t, g, rel, stats[t])
        res = okkt.kkt(A, edges, w, g, X[t], U[t])
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, g, res)
        assert abs(res["kkt"] - stats[t]["kkt"]) <= 1e-8 + 1e-3 * res["kkt"], (res, stats[t])
        assert np.array_equal(lab[t], olabels.labels(X[t], edges)), t
        if not _ambiguous(Xo[t], edges) and not _ambiguous(X[t], edges):
            assert np.array_equal(lab[t], olabels.labels(Xo[t], edges)), t
        assert stats[t]["n_clusters"] == lab[t].max() + 1
    return X, stats


@pytest.mark.parametrize("precision,engine", [(0, 1), (1, 1), (0, 2), (1, 2)])
def test_gmm200_path_matches_oracle(ccm, precision, engine):
    """The n = 200, d = 2 workload on both engines (GRID = 1, BLOCK = 2)."""
    A, _, wl = synth.make_workload("gmm200_d2", 0)
    edges, w, _ = ograph.build_graph(A, wl.k, wl.phi)
    gammas = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    _check_path(ccm, A, edges, w, gammas, precision, engine=engine)


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("seed,n,d,k", [(1, 40, 1, 4), (2, 50, 3, 5), (3, 45, 7, 6),
                                         (4, 60, 17, 5), (5, 33, 64, 4)])
def test_small_random_paths(ccm, seed, n, d, k, engine):
    rng = np.random.default_rng(seed)
    cent = rng.normal(0, 3, size=(3, d))
    A = cent[rng.integers(0, 3, n)] + 0.8 * rng.normal(size=(n, d))
    A[1] = A[0]                                     # a duplicate point
    edges, w, _ = ograph.build_graph(A, k, 0.0)
    w[::7] = 0.0                                    # inert edges
    gammas = np.array([0.0, 0.01, 0.1, 0.5, 2.0, 50.0])
    _check_path(ccm, A, edges, w, gammas, 1, engine=engine)


def test_rejects_bad_input(ccm):
    A, _, wl = synth.make_workload("gmm200_d2", 0, n=30)
    edges, w, _ = ograph.build_graph(A, 4, 0.5)
    At, Et, wt = _to_dev(A, edges, w)
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, Et, wt, [0.1], q=3)           # q = 1 and 2 only
    bad = edges.copy()
    bad[3] = [5, 5]
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, torch.tensor(bad, dtype=torch.int32, device="cuda:0"), wt, [0.1])
    bad = edges.copy()
    bad[0, 1] = 30                                  # out of range
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, torch.tensor(bad, dtype=torch.int32, device="cuda:0"), wt, [0.1])
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, Et, wt, [0.5, 0.1])      # decreasing gammas


def test_deterministic(ccm):
    A, _, wl = synth.make_workload("gmm200_d2", 1, n=120)
    edges, w, _ = ograph.build_graph(A, 8, 0.5)
    At, Et, wt = _to_dev(A, edges, w)
    g = [0.05, 0.3, 1.5]
    for engine in (1, 2):
        X1, L1, _, _ = ccm.solve_path(At, Et, wt, g, engine=engine)
        X2, L2, _, _ = ccm.solve_path(At, Et, wt, g, engine=engine)
        assert torch.equal(X1, X2) and torch.equal(L1, L2)


def test_labels_entry_point(ccm):
    X = np.array([[0.0, 0.0], [0.0, 1e-6], [0.0, 3e-6], [5.0, 5.0], [5.0, 5.0]])
    E = np.array([[0, 1], [1, 2], [2, 3], [3, 4]])
    lab, K = ccm.labels(torch.tensor(X, device="cuda:0"),
                        torch.tensor(E, dtype=torch.int32, device="cuda:0"))
    assert lab.cpu().tolist() == olabels.labels(X, E).tolist() == [0, 0, 1, 2, 2]
    assert K == 3


def _hub_graph(seed, n, d, k):
    """kNN graph plus one hub joined to every other node, one isolated node and
    some inert edges: long rows (d > 128) run the shared-memory ring kernels,
    whose even split of the incidence stream cuts the hub into many parts."""
    rng = np.random.default_rng(seed)
    cent = rng.normal(0, 2, size=(4, d))
    A = cent[rng.integers(0, 4, n)] + rng.normal(size=(n, d))
    edges, w, _ = ograph.build_graph(A[: n - 1], k, 0.0)   # node n-1 stays isolated
    hub = 3
    extra = np.array([[min(hub, j), max(hub, j)] for j in range(n - 1) if j != hub])
    allE = np.concatenate([edges, extra])
    allw = np.concatenate([w, np.full(len(extra), 0.02)])
    key = allE[:, 0] * n + allE[:, 1]
    _, idx = np.unique(key, return_index=True)
    E, wE = allE[idx], allw[idx]
    wE[::11] = 0.0                                          # inert edges
    return A, E, wE


@pytest.mark.parametrize("precision", [1, 0])
def test_long_rows_hub_matches_oracle(ccm, precision):
    A, E, w = _hub_graph(11, 90, 260, 4)
    gammas = np.array([0.5, 5.0, 20.0, 80.0])         # 90, 90, 6, 5 clusters
    X, _ = _check_path(ccm, A, E, w, gammas, precision, engine=1)
    At, Et, wt = _to_dev(A, E, w)
    X1, L1, _, _ = ccm.solve_path(At, Et, wt, gammas, tol=SOLVE_TOL, precision=precision, engine=1)
    X2, L2, _, _ = ccm.solve_path(At, Et, wt, gammas, tol=SOLVE_TOL, precision=precision, engine=1)
    assert torch.equal(X1, X2) and torch.equal(L1, L2)     # split parts sum in a fixed order


@pytest.mark.parametrize("precision", [1, 0])
def test_long_rows_degenerate_graphs(ccm, precision):
    """Long rows (ring kernels) on degenerate graphs: no edges (X = A for every
    gamma), a single node, and one edge between two points (the n = 2 closed
    form: fused iff 2 gamma w >= ||a_1 - a_2||)."""
    rng = np.random.default_rng(21)
    d = 200
    A = rng.normal(size=(50, d))
    At = torch.tensor(A, device="cuda:0")
    E0 = torch.zeros((0, 2), dtype=torch.int32, device="cuda:0")
    w0 = torch.zeros((0,), dtype=torch.float64, device="cuda:0")
    X, lab, _, st = ccm.solve_path(At, E0, w0, [0.0, 1.0, 10.0], tol=SOLVE_TOL,
                                   precision=precision, engine=1)
    assert torch.equal(X[0], At) and torch.equal(X[2], At)
    assert lab[2].cpu().tolist() == list(range(50))
    X1, _, _, _ = ccm.solve_path(At[:1], E0, w0, [0.5], tol=SOLVE_TOL, precision=precision,
                                 engine=1)
    assert torch.equal(X1[0], At[:1])
    a = A[:2]
    gap = np.linalg.norm(a[0] - a[1])
    E1 = torch.tensor([[0, 1]], dtype=torch.int32, device="cuda:0")
    w1 = torch.tensor([1.0], dtype=torch.float64, device="cuda:0")
    gam = [0.25 * gap, 0.75 * gap]          # below and above the fusion threshold gap / 2
    # tight tolerance: the fused pair must end below the 1e-6 label threshold
    X2, lab2, _, _ = ccm.solve_path(At[:2], E1, w1, gam, tol=1e-10, precision=precision,
                                    engine=1)
    X2 = X2.cpu().numpy()
    delta = (a[0] - a[1]) / gap
    want0 = np.stack([a[0] - gam[0] * delta, a[1] + gam[0] * delta])
    want1 = np.tile(a.mean(0), (2, 1))
    assert np.linalg.norm(X2[0] - want0) <= 1e-6 * np.linalg.norm(want0)
    assert np.linalg.norm(X2[1] - want1) <= 1e-6 * np.linalg.norm(want1)
    assert lab2.cpu().tolist() == [[0, 1], [0, 0]]


_SHARED_KERNEL_SCRIPT = r"""
import numpy as np, torch
import paper_2501_15964_b300 as ccm
rng = np.random.default_rng(5)
cent = rng.normal(0, 2, size=(3, 150))
A = cent[rng.integers(0, 3, 40)] + rng.normal(size=(40, 150))
At = torch.tensor(A, device="cuda:0")
E, w, _ = ccm.build_graph(At, 4)
# the FP64 long-row ring kernels need more than 48 KB of dynamic shared memory;
# ADMM and SSNAL launch them from different translation units
_, _, _, st = ccm.solve_path_admm(At, E, w, [1.0], tol=1e-6, precision=0)
assert all(s["status"] == 0 for s in st), st
for q in (2, 1, "inf"):
    _, _, _, st = ccm.solve_path(At, E, w, [0.5, 2.0], q=q, tol=1e-6, precision=0)
    assert all(s["status"] == 0 for s in st), (q, st)
print("ok")
"""


def test_ring_kernels_after_another_solver_in_a_fresh_process(ccm):
    """The ring kernels' shared-memory limit is raised per kernel instance: an
    ADMM solve followed by SSNAL solves (q = 2, 1, inf) on FP64 long rows in a new
    process, where no earlier launch has set anything."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _SHARED_KERNEL_SCRIPT], cwd=root,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


@pytest.mark.parametrize("engine", [1, 2])
def test_iteration_cap_reports_not_converged_with_outputs(ccm, engine):
    """max_outer = 1 cannot reach the tolerance: the call returns
    CCM_ERR_NOT_CONVERGED (status 5), every gamma's status says so, and X, the
    labels and the statistics are still written (X finite, labels equal to the
    oracle's rule on that X, KKT reported above the tolerance)."""
    A, _, wl = synth.make_workload("gmm200_d2", 0)
    E, w, _ = ograph.build_graph(A, wl.k, wl.phi)
    g = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, 6)
    At, Et, wt = _to_dev(A, E, w)
    with pytest.raises(ccm.CCMError) as ei:
        ccm.solve_path(At, Et, wt, g, tol=1e-12, engine=engine, max_outer=1, raise_on_cap=True)
    assert ei.value.status == 5
    X, lab, _, st = ccm.solve_path(At, Et, wt, g, tol=1e-12, engine=engine, max_outer=1)
    X = X.cpu().numpy()
    lab = lab.cpu().numpy()
    assert np.all(np.isfinite(X))
    assert any(s["status"] == 5 for s in st)
    for t in range(len(g)):
        assert st[t]["status"] in (0, 5) and st[t]["outer"] == 1
        assert (st[t]["status"] == 0) == (st[t]["kkt"] <= 1e-12 and st[t]["gap"] <= 1e-12)
        assert np.array_equal(lab[t], olabels.labels(X[t], E))


def test_resume_from_saved_state_equals_full_path(ccm):
    """Checkpoint / resume: solve gamma[:k], save (X, U) of gamma[k-1], then
    solve gamma[k:] from X0 = X, U0 = U (a warm start, which also sends AUTO to
    the grid engine). Both halves equal the uninterrupted path within 1e-6
    relative; the solution of each gamma is unique (strongly convex model,
    Sec. 1), only the iterates differ."""
    A, _, wl = synth.make_workload("gmm200_d2", 1)
    E, w, _ = ograph.build_graph(A, wl.k, wl.phi)
    g = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    At, Et, wt = _to_dev(A, E, w)
    Xf, Lf, _, _ = ccm.solve_path(At, Et, wt, g, tol=SOLVE_TOL)
    k = 9
    X1, L1, U1, _ = ccm.solve_path(At, Et, wt, g[:k], tol=SOLVE_TOL, return_U=True)
    X2, L2, _, st2 = ccm.solve_path(At, Et, wt, g[k:], tol=SOLVE_TOL, X0=X1[-1].contiguous(),
                                    U0=U1[-1].contiguous())
    assert all(s["status"] == 0 for s in st2)
    Xr = torch.cat([X1, X2]).cpu().numpy()
    Xf = Xf.cpu().numpy()
    for t in range(len(g)):
        assert np.linalg.norm(Xr[t] - Xf[t]) <= TOL * np.linalg.norm(Xf[t]), t
    Lr = torch.cat([L1, L2]).cpu().numpy()
    Lf = Lf.cpu().numpy()
    for t in range(len(g)):
        if not _ambiguous(Xf[t], E):
            assert np.array_equal(Lr[t], Lf[t]), t
    with pytest.raises(ccm.CCMError):
        ccm.solve_path(At, Et, wt, g[k:], tol=SOLVE_TOL, X0=X1[-1].contiguous(), engine=2)


@pytest.mark.parametrize("precision", [1, 0])
def test_relabelled_solve_matches_plain_order(ccm, precision):
    """From n = 16,384 nodes the grid engine solves with the nodes grouped by
    connected component (options.relabel = 1, the default) and maps inputs and
    outputs through the permutation, flipping the sign of U rows whose edge
    endpoints swap. The solution is unique (Sec. 1), so X must agree with the
    solve in the caller's order; the oracle's KKT residuals and gap of the
    returned (X, U) check the U rows and their signs; labels agree where no
    edge distance is in the ambiguous band."""
    rng = np.random.default_rng(17)
    n, d = 20000, 3
    cent = rng.normal(0, 4, size=(40, d))
    A = cent[rng.integers(0, 40, n)] + 0.7 * rng.normal(size=(n, d))
    At = torch.tensor(A, device="cuda:0")
    Et, wt, _ = ccm.build_graph(At, 6, 0.0)
    E = Et.cpu().numpy().astype(np.int64)
    w = wt.cpu().numpy()
    g = [0.01, 0.1, 0.6]
    runs = {}
    for rl in (0, 1):
        X, L, U, st = ccm.solve_path(At, Et, wt, g, tol=SOLVE_TOL, return_U=True,
                                     precision=precision, relabel=rl)
        assert all(s["status"] == 0 for s in st)
        runs[rl] = (X.cpu().numpy(), L.cpu().numpy(), U.cpu().numpy())
    for t, gm in enumerate(g):
        X0, L0, _ = runs[0]
        X1, L1, U1 = runs[1]
        assert np.linalg.norm(X1[t] - X0[t]) <= TOL * np.linalg.norm(X0[t]), t
        res = okkt.kkt(A, E, w, gm, X1[t], U1[t])
        assert res["kkt"] <= TOL and res["gap"] <= TOL, (t, res)
        assert np.array_equal(L1[t], olabels.labels(X1[t], E))
        if not _ambiguous(X0[t], E):
            assert np.array_equal(L1[t], L0[t]), t
    # warm start through the maps: U0 rows enter with their signs
    Xa, _, Ua, _ = ccm.solve_path(At, Et, wt, g[:2], tol=SOLVE_TOL, return_U=True,
                                  precision=precision)
    Xb, _, _, stb = ccm.solve_path(At, Et, wt, g[2:], tol=SOLVE_TOL, precision=precision,
                                   X0=Xa[-1].contiguous(), U0=Ua[-1].contiguous())
    assert stb[0]["status"] == 0
    Xb = Xb.cpu().numpy()
    assert np.linalg.norm(Xb[0] - runs[0][0][2]) <= TOL * np.linalg.norm(runs[0][0][2])


@pytest.mark.parametrize("engine", [1, 2])
def test_host_outputs_equal_device_outputs(ccm, engine):
    """X and labels written to pinned (and pageable) host memory by the library
    (each gamma's X copied while the next one solves) equal the device outputs
    bit for bit; U must stay device memory."""
    rng = np.random.default_rng(31)
    n, d = (3000, 5) if engine == 1 else (300, 5)
    cent = rng.normal(0, 4, size=(6, d))
    A = cent[rng.integers(0, 6, n)] + 0.7 * rng.normal(size=(n, d))
    At = torch.tensor(A, device="cuda:0")
    Et, wt, _ = ccm.build_graph(At, 8, 0.0)
    g = [0.01, 0.1, 0.5, 2.0]
    X0, L0, _, st0 = ccm.solve_path(At, Et, wt, g, tol=SOLVE_TOL, engine=engine)
    for pinned in (True, False):
        Xh = torch.empty((len(g), n, d), dtype=torch.float64)
        Lh = torch.empty((len(g), n), dtype=torch.int32)
        if pinned:
            Xh, Lh = Xh.pin_memory(), Lh.pin_memory()
        X1, L1, _, st1 = ccm.solve_path(At, Et, wt, g, tol=SOLVE_TOL, engine=engine,
                                        X_out=Xh, labels_host=Lh)
        assert X1.data_ptr() == Xh.data_ptr() and L1.data_ptr() == Lh.data_ptr()
        assert torch.equal(Xh, X0.cpu()) and torch.equal(Lh, L0.cpu()), pinned
        assert [s["n_clusters"] for s in st1] == [s["n_clusters"] for s in st0]
    E = torch.empty((len(g), Et.shape[0], d), dtype=torch.float64)
    lib = ccm._lib.load_library()
    ctx = ccm.api.default_context(0)
    garr = (ccm._lib.C.c_double * len(g))(*g)
    opt = ccm.api.make_options(engine=engine)
    st = lib.ccm_solve_path(ctx.handle, At.data_ptr(), n, d, Et.data_ptr(), wt.data_ptr(),
                            Et.shape[0], garr, len(g), 2, SOLVE_TOL, ccm._lib.C.byref(opt),
                            X0.data_ptr(), None, E.data_ptr(), None, None)
    assert st == 1  # CCM_ERR_INVALID_ARG: U in host memory
