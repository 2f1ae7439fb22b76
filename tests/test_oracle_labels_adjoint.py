"""Pins for oracle.labels (Sec. 1 cluster rule) and oracle.adjoint."""
import numpy as np

from oracle import adjoint, graph, labels, ssnal


def test_labels_fixture_and_threshold():
    X = np.array([[0.0, 0.0], [0.0, 1e-6], [0.0, 3e-6], [5.0, 5.0], [5.0, 5.0]])
    E = np.array([[0, 1], [1, 2], [2, 3], [3, 4]])
    # (0,1): |d| = 1e-6 -> fused (D = 1e-12 <= 1e-12); (1,2): 2e-6 -> not;
    # (2,3) far; (3,4) equal -> fused
    assert labels.labels(X, E).tolist() == [0, 0, 1, 2, 2]
    # canonical numbering follows the smallest member index
    X2 = X[[3, 0, 1, 4, 2]]
    E2 = np.array([[1, 2], [2, 4], [0, 4], [0, 3]])
    assert labels.labels(X2, E2).tolist() == [0, 1, 1, 0, 2]


def test_labels_gamma_extremes():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(30, 2))
    edges, w, _ = graph.build_graph(A, 4, 0.5)
    assert len(np.unique(labels.labels(A, edges))) == 30
    X, _, _, _ = ssnal.solve(A, edges, w, 1e4, tol=1e-12)
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    ncomp, _ = connected_components(coo_matrix((np.ones(len(edges)), tuple(edges.T)),
                                               shape=(30, 30)), directed=False)
    assert labels.labels(X, edges).max() + 1 == ncomp


def test_adjoint_two_points_closed_form():
    """n = 2, hand-derived derivatives of x1 = a1 - r D/|D|, x2 = a2 + r D/|D|."""
    a = np.array([[1.0, 2.0], [4.0, -2.0]])
    E = np.array([[0, 1]])
    w = np.array([0.8])
    G = np.array([[0.3, -1.2], [0.7, 0.4]])
    for gamma in [0.5, 5.0]:
        X, _, _, _ = ssnal.solve(a, E, w, gamma, tol=1e-13)
        dA, dw = adjoint.vjp_one(a, E, w, gamma, X, G)
        D = a[0] - a[1]
        nD = np.linalg.norm(D)
        s = D / nD
        r = gamma * w[0]
        if 2 * r >= nD:
            wantA = np.tile(G.mean(0), (2, 1))
            wantw = 0.0
        else:
            Pj = (r / nD) * (np.eye(2) - np.outer(s, s))
            g = G[0] - G[1]
            wantA = np.stack([G[0] - Pj @ g, G[1] + Pj @ g])
            wantw = -gamma * s @ g
        np.testing.assert_allclose(dA, wantA, atol=1e-10)
        np.testing.assert_allclose(dw, [wantw], atol=1e-10)


def test_adjoint_matches_central_differences():
    rng = np.random.default_rng(3)
    n, d = 12, 2
    cent = np.array([[0.0, 0.0], [4.0, 0.0], [0.0, 4.0]])
    A = cent[rng.integers(0, 3, n)] + 0.6 * rng.normal(size=(n, d))
    edges, w, _ = graph.build_graph(A, 3, 0.5)
    T = rng.normal(size=(n, d))
    gammas = np.array([0.05, 0.3])

    def loss(Av, wv):
        Xs, _, _ = ssnal.solve_path(Av, edges, wv, gammas, tol=1e-13)
        return sum(np.sum((Xs[t] - T) ** 2) for t in range(len(gammas))), Xs

    L0, Xs = loss(A, w)
    Gs = [2 * (Xs[t] - T) for t in range(len(gammas))]
    dA, dw = adjoint.path_vjp(A, edges, w, gammas, Xs, Gs)
    h = 1e-6
    checked = 0
    for _ in range(6):
        VA = rng.normal(size=A.shape)
        Vw = rng.normal(size=w.shape)
        nrm = np.sqrt(np.sum(VA ** 2) + np.sum(Vw ** 2))
        VA /= nrm
        Vw /= nrm
        Lp, Xp = loss(A + h * VA, w + h * Vw)
        Lm, Xm = loss(A - h * VA, w - h * Vw)
        same = all(np.array_equal(labels.labels(Xp[t], edges), labels.labels(Xm[t], edges))
                   for t in range(len(gammas)))
        if not same:
            continue                                   # crosses a fusion event
        fd = (Lp - Lm) / (2 * h)
        an = np.sum(dA * VA) + np.sum(dw * Vw)
        assert abs(fd - an) <= 1e-4 * (1 + abs(an))
        checked += 1
    assert checked >= 4
