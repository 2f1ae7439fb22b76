"""Pins for oracle.graph (kNN graph and weights of model CCM, Sec. 1 / Sec. 2.2)."""
import os

import numpy as np
import pytest

import synth
from oracle import graph

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    rows = [ln.split() for ln in open(os.path.join(GOLD, name))
            if ln.strip() and not ln.startswith("#")]
    n, d, k = map(int, rows[0])
    A = np.array(rows[1:1 + n], dtype=np.float64).reshape(n, d)
    return n, d, k, A, rows[1 + n:]


def test_knn_tie_fixture():
    n, d, k, A, rest = _read_fixture("knn_ties.txt")
    expect = np.array(rest, dtype=np.int64).reshape(n, k)
    assert np.array_equal(graph.knn(A, k), expect)


def test_lower_median_fixture():
    n, d, k, A, rest = _read_fixture("median_phi.txt")
    exp_edges = np.array(rest[:3], dtype=np.int64)
    exp_phi = float(rest[3][0])
    edges, w, phi = graph.build_graph(A, k, 0.0)
    assert np.array_equal(edges, exp_edges)
    assert phi == exp_phi
    np.testing.assert_allclose(w, np.exp(-exp_phi * np.array([1.0, 4.0, 16.0])), rtol=0)


def test_canonical_distance_symmetric_and_exact():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(40, 7))
    D = graph.canonical_sqdist_rows(A, np.arange(40))
    assert np.array_equal(D, D.T)                # bitwise symmetric
    assert np.all(np.diag(D) == 0)
    # agrees with a mathematically identical formula to rounding
    ref = ((A[:, None, :] - A[None, :, :]) ** 2).sum(-1)
    np.testing.assert_allclose(D, ref, rtol=1e-14, atol=1e-14)


def test_knn_matches_sklearn_away_from_ties():
    sk = pytest.importorskip("sklearn.neighbors")
    A, _, _ = synth.make_workload("gmm200_d2", 0)
    k = 10
    mine = graph.knn(A, k)
    nn = sk.NearestNeighbors(n_neighbors=k + 1, algorithm="brute").fit(A)
    dist, idx = nn.kneighbors(A)
    D = graph.canonical_sqdist_rows(A, np.arange(A.shape[0]))
    checked = 0
    for i in range(A.shape[0]):
        row = np.sort(np.delete(D[i], i))
        if row[k] - row[k - 1] < 1e-9 * (1 + row[k]):
            continue                                     # near tie: skip
        theirs = [j for j in idx[i] if j != i][:k]
        assert set(theirs) == set(mine[i])
        checked += 1
    assert checked > 150


def test_symmetrize_union_properties():
    A, _, wl = synth.make_workload("gmm200_d2", 0)
    nbrs = graph.knn(A, wl.k)
    edges = graph.symmetrize(nbrs)
    n, k = nbrs.shape
    m = edges.shape[0]
    assert n * k / 2 <= m <= n * k
    assert np.all(edges[:, 0] < edges[:, 1])
    key = edges[:, 0] * n + edges[:, 1]
    assert np.all(np.diff(key) > 0)                      # sorted, unique
    es = set(map(tuple, edges.tolist()))
    for i in range(n):                                   # every directed pair present
        for j in nbrs[i]:
            assert (min(i, j), max(i, j)) in es
    for (a, b) in es:                                    # and nothing else
        assert b in nbrs[a] or a in nbrs[b]


def test_weights_given_phi():
    D = np.array([0.0, 1.0, 2.5])
    w, phi = graph.weights(D, 0.5)
    assert phi == 0.5
    np.testing.assert_allclose(w, np.exp(-0.5 * D), rtol=0)
    with pytest.raises(ValueError):
        graph.weights(np.zeros(3), 0.0)
