"""GPU parity of ccm_path_vjp (implicit differentiation of the path; not in
the paper) against the dense float64 oracle gradient and central differences.

Tolerances: the GPU and the oracle differentiate at their own solutions,
which agree to about 1e-7 relative, so the gradients agree to about 1e-5;
central differences of GPU solves at step 1e-4 agree to about 1e-4. Directions
whose +-h solves change the fusion pattern are skipped (counted).
"""
import numpy as np
import pytest

import synth
from oracle import adjoint as oadj
from oracle import graph as ograph
from oracle import labels as olabels
from oracle import ssnal as ossnal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    import paper_2501_15964_b300 as m
    return m


def _dev(*arrs):
    out = []
    for a in arrs:
        a = np.asarray(a)
        out.append(torch.tensor(a, dtype=torch.int32 if a.dtype.kind == "i" else torch.float64,
                                device="cuda:0"))
    return out


def _gpu_grad(ccm, A, E, w, gammas, T, tol=1e-10):
    At, Et, wt = _dev(A, E, w)
    X, L, _, st = ccm.solve_path(At, Et, wt, gammas, tol=tol, precision=0, engine=1)
    G = 2.0 * (X - torch.tensor(T, device="cuda:0"))
    dA, dw = ccm.path_vjp(At, Et, wt, gammas, X, G)
    return X.cpu().numpy(), L.cpu().numpy(), dA.cpu().numpy(), dw.cpu().numpy()


@pytest.mark.parametrize("seed,n,d,k", [(0, 40, 3, 5), (1, 60, 8, 6), (2, 30, 1, 4)])
def test_vjp_matches_dense_oracle(ccm, seed, n, d, k):
    rng = np.random.default_rng(seed)
    cent = rng.normal(0, 3, size=(3, d))
    A = cent[rng.integers(0, 3, n)] + 0.7 * rng.normal(size=(n, d))
    E, w, _ = ograph.build_graph(A, k, 0.0)
    T = rng.normal(size=(n, d))
    gammas = np.array([0.02, 0.2, 1.0, 5.0])
    Xo, _, _ = ossnal.solve_path(A, E, w, gammas, tol=1e-12)
    Go = [2 * (Xo[t] - T) for t in range(len(gammas))]
    dAo, dwo = oadj.path_vjp(A, E, w, gammas, Xo, Go)
    X, L, dA, dw = _gpu_grad(ccm, A, E, w, gammas, T)
    for t in range(len(gammas)):
        assert np.array_equal(L[t], olabels.labels(Xo[t], E)), t
    assert np.linalg.norm(dA - dAo) <= 2e-5 * np.linalg.norm(dAo)
    assert np.linalg.norm(dw - dwo) <= 2e-5 * max(np.linalg.norm(dwo), 1e-12)


def test_vjp_central_differences(ccm):
    rng = np.random.default_rng(4)
    n, d = 50, 4
    cent = rng.normal(0, 3, size=(4, d))
    A = cent[rng.integers(0, 4, n)] + 0.8 * rng.normal(size=(n, d))
    E, w, _ = ograph.build_graph(A, 5, 0.0)
    T = rng.normal(size=(n, d))
    gammas = np.array([0.05, 0.5])
    X, L, dA, dw = _gpu_grad(ccm, A, E, w, gammas, T, tol=1e-11)

    def loss(Av, wv):
        At, Et, wt = _dev(Av, E, wv)
        Xv, Lv, _, _ = ccm.solve_path(At, Et, wt, gammas, tol=1e-11, precision=0, engine=1)
        Xv = Xv.cpu().numpy()
        return sum(np.sum((Xv[t] - T) ** 2) for t in range(len(gammas))), Lv.cpu().numpy()

    h = 1e-4
    ok = skipped = 0
    for _ in range(20):
        VA = rng.normal(size=A.shape)
        Vw = rng.normal(size=w.shape)
        nrm = np.sqrt(np.sum(VA ** 2) + np.sum(Vw ** 2))
        VA, Vw = VA / nrm, Vw / nrm
        Lp, lp = loss(A + h * VA, w + h * Vw)
        Lm, lm = loss(A - h * VA, w - h * Vw)
        if not (np.array_equal(lp, L) and np.array_equal(lm, L)):
            skipped += 1
            continue
        fd = (Lp - Lm) / (2 * h)
        an = np.sum(dA * VA) + np.sum(dw * Vw)
        assert abs(fd - an) <= 1e-4 * (1 + abs(an)), (fd, an)
        ok += 1
    assert ok >= 15, (ok, skipped)


def test_vjp_dense_oracle_n500_d64(ccm):
    """The adjoint workload's recipe (n = 500 points, d = 64, k = 10, phi =
    1/median) at two gammas inside its grid's fusion range, where the oracle's
    solution has 30 and 23 clusters joined by 99 and 30 unfused edges: the
    dense reduced system stays (K d)^2 <= 1920^2 while every term of the adjoint
    (the M block, the c_l (I - s s^T) blocks of the unfused edges, dL/dw on
    them) is exercised. The fusion margins at these gammas (smallest unfused
    distance 0.011, largest fused about 1e-8 in the oracle's solution) keep
    the labels clear of the 1e-6 rule."""
    A, _, wl = synth.make_workload("gmm20k_d64", 0, n=500)
    E, w, _ = ograph.build_graph(A, wl.k, wl.phi)
    T = synth.adjoint_target(0, 500, 64)
    gammas = np.array([3.1, 3.7])
    Xo, _, _ = ossnal.solve_path(A, E, w, gammas, tol=1e-11)
    n_unfused = []
    for t in range(len(gammas)):
        lab = olabels.labels(Xo[t], E)
        assert 20 < lab.max() + 1 <= 250
        n_unfused.append(int(np.sum(lab[E[:, 0]] != lab[E[:, 1]])))
    assert min(n_unfused) > 0, n_unfused
    Go = [2 * (Xo[t] - T) for t in range(len(gammas))]
    dAo, dwo = oadj.path_vjp(A, E, w, gammas, Xo, Go)
    assert np.count_nonzero(dwo) > 0
    X, L, dA, dw = _gpu_grad(ccm, A, E, w, gammas, T)
    for t in range(len(gammas)):
        assert np.array_equal(L[t], olabels.labels(Xo[t], E)), t
    assert np.linalg.norm(dA - dAo) <= 1e-5 * np.linalg.norm(dAo)
    assert np.linalg.norm(dw - dwo) <= 1e-5 * np.linalg.norm(dwo)
    # dL/dw is supported exactly on the unfused edges of either gamma
    assert np.array_equal(np.nonzero(dw)[0], np.nonzero(dwo)[0])


def test_autograd_function_matches_vjp(ccm):
    rng = np.random.default_rng(9)
    n, d = 30, 2
    A = rng.normal(size=(n, d)) * 3
    E, w, _ = ograph.build_graph(A, 4, 0.0)
    At, Et, wt = _dev(A, E, w)
    At.requires_grad_(True)
    wt.requires_grad_(True)
    g = [0.1, 1.0]
    X = ccm.CCMPath.apply(At, wt, Et, g, 1e-10)
    T = torch.tensor(rng.normal(size=(n, d)), device="cuda:0")
    loss = ((X - T) ** 2).sum()
    loss.backward()
    dA, dw = ccm.path_vjp(At.detach(), Et, wt.detach(), g, X.detach(), 2 * (X.detach() - T))
    assert torch.allclose(At.grad, dA, rtol=1e-12, atol=1e-12)
    assert torch.allclose(wt.grad, dw, rtol=1e-12, atol=1e-12)
