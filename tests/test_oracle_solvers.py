"""Pins for the oracle solvers of model CCM (Sec. 1) and the gap of Sec. 4.

Each test checks the oracle against something other than itself: a closed
form, an exact combinatorial solution, an invariance, a bound, or a second,
independent algorithm.
"""
import numpy as np
import pytest

from oracle import admm, exact1d, graph, kkt, labels, ssnal


def _small_problem(seed=0, n=40, d=3, k=5, phi=0.5):
    rng = np.random.default_rng(seed)
    cent = rng.normal(0, 3, size=(3, d))
    A = cent[rng.integers(0, 3, n)] + 0.7 * rng.normal(size=(n, d))
    edges, w, _ = graph.build_graph(A, k, phi)
    return A, edges, w


def test_two_points_closed_form():
    """n = 2: x1 = a1 - r D/|D|, x2 = a2 + r D/|D| until 2r >= |D|, then the mean."""
    a = np.array([[1.0, 2.0], [4.0, -2.0]])                 # |D| = 5
    E = np.array([[0, 1]])
    w = np.array([0.8])
    for gamma in [0.1, 1.0, 3.0, 3.2, 10.0]:
        r = gamma * w[0]
        D = a[0] - a[1]
        nD = np.linalg.norm(D)
        if 2 * r >= nD:
            want = np.tile(a.mean(0), (2, 1))
        else:
            want = np.stack([a[0] - r * D / nD, a[1] + r * D / nD])
        X, U, _, info = ssnal.solve(a, E, w, gamma, tol=1e-13)
        np.testing.assert_allclose(X, want, atol=1e-11)
        assert info["kkt"] <= 1e-12


def test_gamma_zero_is_identity():
    A, edges, w = _small_problem()
    X, U, _, info = ssnal.solve(A, edges, w, 0.0)
    assert np.array_equal(X, A)
    assert np.all(U == 0)
    assert len(np.unique(labels.labels(X, edges))) == A.shape[0]


@pytest.mark.parametrize("gamma", [0.002, 0.01, 0.03, 0.08, 0.5])
def test_exact_1d_complete_graph(gamma):
    """SSNAL and ADMM reach the certified exact 1-D solution."""
    a = np.random.default_rng(1).normal(size=(20, 1))
    E = exact1d.complete_graph(20)
    w = np.ones(E.shape[0])
    xe = exact1d.solve(a[:, 0], gamma)
    X, _, _, _ = ssnal.solve(a, E, w, gamma, tol=1e-12)
    Xa, _, _ = admm.solve(a, E, w, gamma, tol=1e-11, max_iter=20000)
    np.testing.assert_allclose(X[:, 0], xe, atol=1e-10)
    np.testing.assert_allclose(Xa[:, 0], xe, atol=1e-9)


def test_path_graph_fusion_threshold():
    """Tree graph: full fusion starts exactly at gamma = max_l |u_l| / w_l with
    B^T U = A - mean(A) solved along the chain."""
    rng = np.random.default_rng(2)
    n, d = 8, 2
    A = rng.normal(size=(n, d))
    E = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1)
    w = rng.uniform(0.5, 1.5, size=n - 1)
    u = np.cumsum(A - A.mean(0), axis=0)[:-1]        # u_l = sum_{i<=l} (a_i - mean)
    g_fuse = np.max(np.linalg.norm(u, axis=1) / w)
    X, _, _, _ = ssnal.solve(A, E, w, g_fuse * 1.001, tol=1e-12)
    np.testing.assert_allclose(X, np.tile(A.mean(0), (n, 1)), atol=1e-9)
    X, _, _, _ = ssnal.solve(A, E, w, g_fuse * 0.98, tol=1e-12)
    assert np.max(np.linalg.norm(X - X.mean(0), axis=1)) > 1e-4


def test_large_gamma_gives_component_centroids():
    """Sec. 1: on a connected graph every x_i tends to the centroid; per
    component when the graph is disconnected."""
    A, edges, w = _small_problem(seed=4, n=30, d=2, k=4)
    # add a far, separate triangle (its own component)
    far = np.array([[50.0, 50.0], [51.0, 50.0], [50.0, 51.5]])
    A2 = np.vstack([A, far])
    n = A.shape[0]
    E2 = np.vstack([edges, np.array([[n, n + 1], [n, n + 2], [n + 1, n + 2]])])
    w2 = np.concatenate([w, [0.5, 0.5, 0.5]])
    X, _, _, _ = ssnal.solve(A2, E2, w2, 1e4, tol=1e-12)
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    _, comp = connected_components(coo_matrix((np.ones(len(E2)), (E2[:, 0], E2[:, 1])),
                                              shape=(n + 3, n + 3)), directed=False)
    for c in np.unique(comp):
        sel = comp == c
        np.testing.assert_allclose(X[sel], np.tile(A2[sel].mean(0), (sel.sum(), 1)), atol=1e-8)


def test_invariances_and_mean_preservation():
    A, edges, w = _small_problem(seed=5, n=30, d=3, k=5)
    g = 0.3
    X, _, _, _ = ssnal.solve(A, edges, w, g, tol=1e-12)
    np.testing.assert_allclose(X.sum(0), A.sum(0), atol=1e-9)           # sum x = sum a
    c = np.array([3.0, -1.0, 2.0])
    Xt, _, _, _ = ssnal.solve(A + c, edges, w, g, tol=1e-12)
    np.testing.assert_allclose(Xt, X + c, atol=1e-9)                     # translation
    Q, _ = np.linalg.qr(np.random.default_rng(6).normal(size=(3, 3)))
    Xr, _, _, _ = ssnal.solve(A @ Q, edges, w, g, tol=1e-12)
    np.testing.assert_allclose(Xr, X @ Q, atol=1e-9)                     # rotation
    s = 2.5
    Xs, _, _, _ = ssnal.solve(s * A, edges, w, s * g, tol=1e-12)
    np.testing.assert_allclose(Xs, s * X, atol=1e-8)                     # scaling
    perm = np.random.default_rng(7).permutation(A.shape[0])
    inv = np.argsort(perm)
    Ep = np.sort(inv[edges], axis=1)
    order = np.lexsort((Ep[:, 1], Ep[:, 0]))
    Xp, _, _, _ = ssnal.solve(A[perm], Ep[order], w[order], g, tol=1e-12)
    np.testing.assert_allclose(Xp, X[perm], atol=1e-9)                   # permutation


def test_continuity_bound_along_path():
    """|X(g1) - X(g2)| <= |g1 - g2| / g2 * |A - X(g2)| (from monotonicity of the
    subdifferential; Sec. 1 states continuity in gamma)."""
    A, edges, w = _small_problem(seed=8, n=30, d=2, k=5)
    gam = np.array([0.05, 0.06, 0.2, 0.21, 1.0])
    Xs, _, _ = ssnal.solve_path(A, edges, w, gam, tol=1e-12)
    for t in range(len(gam) - 1):
        lhs = np.linalg.norm(Xs[t] - Xs[t + 1])
        rhs = (gam[t + 1] - gam[t]) / gam[t + 1] * np.linalg.norm(A - Xs[t + 1])
        assert lhs <= rhs * (1 + 1e-6) + 1e-9


def test_ssnal_matches_admm():
    A, edges, w = _small_problem(seed=9, n=30, d=2, k=5)
    for g in [0.05, 0.3, 2.0]:
        X, _, _, info = ssnal.solve(A, edges, w, g, tol=1e-12)
        Xa, _, ra = admm.solve(A, edges, w, g, tol=1e-11, max_iter=50000)
        assert info["kkt"] <= 1e-11
        np.testing.assert_allclose(X, Xa, atol=1e-8)


def test_weak_duality_and_gap():
    """f_d(U) <= f_p(X) for every X and every feasible U (Sec. 4 gap is >= 0)."""
    A, edges, w = _small_problem(seed=10, n=25, d=2, k=4)
    rng = np.random.default_rng(11)
    g = 0.4
    r = g * w
    for _ in range(20):
        X = A + rng.normal(size=A.shape)
        U = rng.normal(size=(edges.shape[0], 2))
        U *= (r * rng.uniform(0, 1, size=r.size) / np.linalg.norm(U, axis=1))[:, None]
        res = kkt.kkt(A, edges, w, g, X, U)
        assert res["fd"] <= res["fp"] + 1e-12
    X, U, _, info = ssnal.solve(A, edges, w, g, tol=1e-12)
    res = kkt.kkt(A, edges, w, g, X, U)
    assert res["gap"] <= 1e-11 and res["dual_infeas"] <= 1e-12


def test_planted_sign_error_is_caught(monkeypatch):
    """A plausible mistake (wrong sign of B^T in the gradient) must fail a pin."""
    def bad_eval(X, A, U, B, r, sigma, q=2):
        Y = U + sigma * (B @ X)
        ny = np.sqrt(np.sum(Y * Y, axis=1))
        inside = ny <= r
        h = np.where(inside, 0.5 * ny * ny, r * ny - 0.5 * r * r)
        phi = 0.5 * np.sum((X - A) ** 2) + np.sum(h) / sigma
        scale = np.ones_like(ny)
        scale[~inside] = r[~inside] / ny[~inside]
        PiY = Y * scale[:, None]
        return phi, X - A - B.T @ PiY, PiY, Y, ny
    monkeypatch.setattr(ssnal, "_eval", bad_eval)
    a = np.array([[1.0, 2.0], [4.0, -2.0]])
    X, _, _, _ = ssnal.solve(a, np.array([[0, 1]]), np.array([0.8]), 1.0, tol=1e-12,
                             max_outer=20)
    want = np.stack([a[0] - 0.8 * (a[0] - a[1]) / 5, a[1] + 0.8 * (a[0] - a[1]) / 5])
    assert not np.allclose(X, want, atol=1e-6)


# ---------------------------------------------------------------- q = 1
def test_two_points_closed_form_q1():
    """n = 2, q = 1: x1 - x2 = soft(a1 - a2, 2 r) per coordinate, x1 + x2 = a1 + a2."""
    a = np.array([[1.0, 2.0, 0.5], [4.0, -2.0, 0.3]])
    E = np.array([[0, 1]])
    w = np.array([0.8])
    for gamma in [0.05, 0.5, 1.0, 3.0]:
        r = gamma * w[0]
        D = a[0] - a[1]
        delta = np.sign(D) * np.maximum(np.abs(D) - 2 * r, 0.0)
        mid = a.mean(0)
        want = np.stack([mid + 0.5 * delta, mid - 0.5 * delta])
        X, U, _, info = ssnal.solve(a, E, w, gamma, tol=1e-13, q=1)
        np.testing.assert_allclose(X, want, atol=1e-11)
        assert info["kkt"] <= 1e-12
        res = kkt.kkt(a, E, w, gamma, X, U, q=1)
        assert res["dual_infeas"] <= 1e-12


@pytest.mark.parametrize("gamma", [0.005, 0.03, 0.2])
def test_q1_complete_graph_is_three_exact_1d_paths(gamma):
    """q = 1 separates by coordinate: on the complete graph with unit weights each
    column is the certified exact 1-D solution of that column."""
    a = np.random.default_rng(4).normal(size=(16, 3))
    E = exact1d.complete_graph(16)
    w = np.ones(E.shape[0])
    X, _, _, info = ssnal.solve(a, E, w, gamma, tol=1e-12, q=1)
    for k in range(3):
        np.testing.assert_allclose(X[:, k], exact1d.solve(a[:, k], gamma), atol=1e-10)


def test_ssnal_matches_admm_q1():
    A, edges, w = _small_problem(seed=12, n=30, d=3, k=5)
    for g in [0.05, 0.4, 2.0]:
        X, _, _, info = ssnal.solve(A, edges, w, g, tol=1e-12, q=1)
        Xa, _, ra = admm.solve(A, edges, w, g, tol=1e-11, max_iter=50000, q=1)
        assert info["kkt"] <= 1e-11
        np.testing.assert_allclose(X, Xa, atol=1e-8)


def test_weak_duality_q1():
    """f_d(U) <= f_p(X) for every X and every U with ||u_l||_inf <= r_l."""
    A, edges, w = _small_problem(seed=13, n=25, d=3, k=4)
    rng = np.random.default_rng(14)
    g = 0.4
    r = g * w
    for _ in range(20):
        X = A + rng.normal(size=A.shape)
        U = rng.uniform(-1, 1, size=(edges.shape[0], 3)) * r[:, None]
        res = kkt.kkt(A, edges, w, g, X, U, q=1)
        assert res["fd"] <= res["fp"] + 1e-12
        assert res["dual_infeas"] == 0.0


# ---------------------------------------------------------------- q = inf
def _vi_violation(v, u, r):
    """Largest <v - u, e - u> over the 2d vertices e = +-r e_k of the l1 ball.

    u is the projection of v onto the ball iff u is in the ball and this is <= 0
    (the ball is the convex hull of its vertices, so checking the variational
    inequality at the vertices checks it everywhere)."""
    g = v - u
    worst = -np.inf
    for k in range(v.size):
        for sgn in (1.0, -1.0):
            e = np.zeros_like(v)
            e[k] = sgn * r
            worst = max(worst, float(g @ (e - u)))
    return worst


def test_l1ball_projection_variational_inequality():
    rng = np.random.default_rng(21)
    for trial in range(300):
        d = int(rng.integers(1, 13))
        v = rng.normal(size=d) * rng.choice([0.1, 1.0, 10.0])
        if trial % 5 == 0:   # ties and zeros
            v = np.round(v) + 0.0
        r = float(rng.uniform(0.0, 1.5) * max(np.sum(np.abs(v)), 1e-3))
        u = kkt.proj_l1ball(v[None, :], np.array([r]))[0]
        scale = 1.0 + np.sum(np.abs(v)) ** 2
        assert np.sum(np.abs(u)) <= r * (1 + 1e-12) + 1e-15
        if np.sum(np.abs(v)) <= r:
            assert np.array_equal(u, v)
        else:
            assert _vi_violation(v, u, r) <= 1e-12 * scale


def test_l1ball_vi_catches_planted_threshold_error():
    """A plausible mistake (dividing by rho + 1 instead of rho) fails the pin above."""
    v = np.array([3.0, -1.0, 0.5, 2.0])
    r = 2.0
    mu = np.sort(np.abs(v))[::-1]
    cs = np.cumsum(mu)
    j = np.arange(1, 5)
    rho = int(np.nonzero(mu * j > cs - r)[0][-1]) + 1
    bad = np.sign(v) * np.maximum(np.abs(v) - (cs[rho - 1] - r) / (rho + 1), 0.0)
    assert _vi_violation(v, bad, r) > 1e-6 or np.sum(np.abs(bad)) > r * (1 + 1e-9)


def test_linf_prox_and_projection_at_d1():
    """d = 1: the l1 ball is [-r, r] and prox of r|.| is the soft threshold."""
    v = np.array([[-3.0], [-0.2], [0.0], [0.7], [5.0]])
    r = np.array([1.0, 1.0, 0.5, 0.5, 2.0])
    np.testing.assert_array_equal(kkt.proj_l1ball(v, r)[:, 0], np.clip(v[:, 0], -r, r))
    np.testing.assert_array_equal(kkt.prox_linf(v, r)[:, 0],
                                  np.sign(v[:, 0]) * np.maximum(np.abs(v[:, 0]) - r, 0.0))


def test_linf_jacobian_matches_finite_differences():
    """diag(mask) - s s^T (the oracle's P_l for q = inf) is the derivative of the
    l1-ball projection away from its kinks."""
    rng = np.random.default_rng(22)
    for _ in range(40):
        d = int(rng.integers(2, 9))
        y = rng.normal(size=d) * 2.0
        r = float(rng.uniform(0.2, 1.2) * np.sum(np.abs(y)))
        pi = kkt.proj_l1ball(y[None, :], np.array([r]))
        mask, svec = ssnal._linf_parts(y[None, :], pi, np.array([r]))
        P = np.diag(mask[0]) - np.outer(svec[0], svec[0])
        h = 1e-7
        J = np.zeros((d, d))
        for k in range(d):
            e = np.zeros(d)
            e[k] = h
            J[:, k] = (kkt.proj_l1ball((y + e)[None, :], np.array([r]))[0]
                       - kkt.proj_l1ball((y - e)[None, :], np.array([r]))[0]) / (2 * h)
        np.testing.assert_allclose(P, J, atol=1e-6)


def test_two_points_closed_form_qinf():
    """n = 2, q = inf, w = 1, a1 - a2 = (4, 1): the penalty r||x1 - x2||_inf first
    shrinks only the larger coordinate of the difference (by 2r) until the two
    coordinates are equal (2r = 3), then both together, and the points fuse at
    2r = ||a1 - a2||_1 = 5. Differences by hand: gamma = 1 -> (2, 1),
    gamma = 2 -> (0.5, 0.5), gamma = 3 -> (0, 0); the mean (3, 0.5) stays."""
    a = np.array([[5.0, 1.0], [1.0, 0.0]])
    E = np.array([[0, 1]])
    w = np.array([1.0])
    mid = np.array([3.0, 0.5])
    for gamma, z in [(1.0, (2.0, 1.0)), (2.0, (0.5, 0.5)), (3.0, (0.0, 0.0))]:
        z = np.array(z)
        X, U, _, info = ssnal.solve(a, E, w, gamma, tol=1e-13, q=np.inf)
        np.testing.assert_allclose(X, np.stack([mid + z / 2, mid - z / 2]), atol=1e-11)
        assert info["kkt"] <= 1e-12
        assert kkt.kkt(a, E, w, gamma, X, U, q=np.inf)["dual_infeas"] <= 1e-12
    # the same with the larger coordinate negative and in second place
    b = np.array([[1.0, -3.0], [0.0, 1.0]])           # a1 - a2 = (1, -4)
    X, _, _, _ = ssnal.solve(b, E, w, 1.0, tol=1e-13, q=np.inf)
    np.testing.assert_allclose(X[0] - X[1], [1.0, -2.0], atol=1e-11)


@pytest.mark.parametrize("gamma", [0.01, 0.05, 0.3])
def test_qinf_in_one_dimension_is_the_exact_1d_path(gamma):
    """d = 1: every q-norm is |.|, so q = inf reduces to the certified exact 1-D path."""
    a = np.random.default_rng(23).normal(size=(14, 1))
    E = exact1d.complete_graph(14)
    w = np.ones(E.shape[0])
    X, _, _, info = ssnal.solve(a, E, w, gamma, tol=1e-12, q=np.inf)
    np.testing.assert_allclose(X[:, 0], exact1d.solve(a[:, 0], gamma), atol=1e-10)


def test_ssnal_matches_admm_qinf():
    A, edges, w = _small_problem(seed=24, n=30, d=3, k=5)
    for g in [0.05, 0.4, 2.0]:
        X, _, _, info = ssnal.solve(A, edges, w, g, tol=1e-12, q=np.inf)
        Xa, _, ra = admm.solve(A, edges, w, g, tol=1e-11, max_iter=50000, q=np.inf)
        assert info["kkt"] <= 1e-11
        np.testing.assert_allclose(X, Xa, atol=1e-8)


def test_weak_duality_qinf():
    """f_d(U) <= f_p(X) for every X and every U with ||u_l||_1 <= r_l."""
    A, edges, w = _small_problem(seed=25, n=25, d=3, k=4)
    rng = np.random.default_rng(26)
    g = 0.4
    r = g * w
    for _ in range(20):
        X = A + rng.normal(size=A.shape)
        U = rng.normal(size=(edges.shape[0], 3))
        U *= (rng.uniform(0, 1, size=edges.shape[0]) * r / np.sum(np.abs(U), axis=1))[:, None]
        res = kkt.kkt(A, edges, w, g, X, U, q=np.inf)
        assert res["fd"] <= res["fp"] + 1e-12
        assert res["dual_infeas"] == 0.0


# ---------------------------------------------------------------- q = 1 and q = inf
@pytest.mark.parametrize("q", [1, np.inf])
def test_separable_norms_invariances(q):
    """For q = 1 and q = inf: sum x = sum a, translation and scaling equivariance,
    and equivariance under signed permutations of the coordinates (the symmetry
    group of both norms; a general rotation is not one of them)."""
    A, edges, w = _small_problem(seed=41, n=24, d=3, k=4)
    g = 0.3
    X, _, _, _ = ssnal.solve(A, edges, w, g, tol=1e-12, q=q)
    np.testing.assert_allclose(X.sum(0), A.sum(0), atol=1e-9)
    c = np.array([3.0, -1.0, 2.0])
    Xt, _, _, _ = ssnal.solve(A + c, edges, w, g, tol=1e-12, q=q)
    np.testing.assert_allclose(Xt, X + c, atol=1e-9)
    s = 2.5
    Xs, _, _, _ = ssnal.solve(s * A, edges, w, s * g, tol=1e-12, q=q)
    np.testing.assert_allclose(Xs, s * X, atol=1e-8)
    S = np.array([[0.0, -1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])  # signed permutation
    Xq, _, _, _ = ssnal.solve(A @ S, edges, w, g, tol=1e-12, q=q)
    np.testing.assert_allclose(Xq, X @ S, atol=1e-9)


@pytest.mark.parametrize("q", [1, np.inf])
def test_separable_norms_large_gamma_centroids(q):
    """Large gamma fuses each connected component to its centroid for every norm."""
    A, edges, _ = _small_problem(seed=42, n=20, d=2, k=4)
    w = np.ones(edges.shape[0])      # unit weights: gamma = 100 is far past full fusion
    X, _, _, info = ssnal.solve(A, edges, w, 100.0, tol=1e-12, q=q)
    assert info["kkt"] <= 1e-11
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    n = A.shape[0]
    _, comp = connected_components(coo_matrix((np.ones(len(edges)), (edges[:, 0], edges[:, 1])),
                                              shape=(n, n)), directed=False)
    for c in np.unique(comp):
        sel = comp == c
        np.testing.assert_allclose(X[sel], np.tile(A[sel].mean(0), (sel.sum(), 1)), atol=1e-8)
