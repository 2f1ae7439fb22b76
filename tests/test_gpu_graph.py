"""GPU parity of ccm_build_graph against the oracle (kNN graph and weights of
model CCM, Sec. 1 / Sec. 2.2): edge sets bit-exact, phi bit-exact, weights
within 2 ulp (libm exp vs CUDA exp)."""
import os

import numpy as np
import pytest

import synth
from oracle import graph as ograph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    import paper_2501_15964_b300 as m
    return m


def _gpu_graph(ccm, A, k, phi):
    At = torch.tensor(A, device="cuda:0")
    E, w, ph = ccm.build_graph(At, k, phi)
    return E.cpu().numpy().astype(np.int64), w.cpu().numpy(), ph


def _check(ccm, A, k, phi):
    E, w, ph = _gpu_graph(ccm, A, k, phi)
    Eo, wo, pho = ograph.build_graph(A, k, phi)
    assert np.array_equal(E, Eo)
    assert ph == pho
    # 2 ulp for normal results; below the normal range (2.2e-308) exp results
    # are subnormal and keep fewer significant bits, so compare absolutely there
    np.testing.assert_allclose(w, wo, rtol=5e-16, atol=1e-300)
    return E


@pytest.mark.parametrize("name,n,phi", [("gmm200_d2", None, 0.5), ("gmm200_d2", None, 0.0),
                                        ("gmm20k_d64", 700, 0.0), ("gmm200k_d50", 1500, 0.5)])
def test_graph_matches_oracle(ccm, name, n, phi):
    A, _, wl = synth.make_workload(name, 0, n=n)
    _check(ccm, A, wl.k, phi)


def test_graph_mnist_like_subsample(ccm):
    A, _, wl = synth.make_workload("mnist10k_d784", 0, n=1000)
    _check(ccm, A, 10, 0.0)
    assert ccm.last_graph_info()["candidates"] == "simt"   # d > 128: CUDA-core tiles


@pytest.mark.parametrize("d", [1, 2, 7, 16, 31, 33, 50, 64, 100, 128])
def test_tensor_core_candidates_match_oracle(ccm, d):
    """d <= 128: candidates from the tcgen05 TF32 Gram form (three-product
    split), re-ranked in float64 under its error bound; the edge set must be the
    oracle's exactly, and the bound must certify (nearly) every row so that the
    exhaustive fallback stays rare. n = 700 spans several 128-row tiles and a
    ragged last tile."""
    rng = np.random.default_rng(100 + d)
    n = 700
    cent = rng.normal(0, 3, size=(6, d))
    A = cent[rng.integers(0, 6, n)] + rng.normal(size=(n, d))
    _check(ccm, A, 10, 0.0)
    info = ccm.last_graph_info()
    assert info["candidates"] == "tensor" and info["per_row"] == 32, info
    assert info["rows_exhaustive"] <= n // 100, info


@pytest.mark.parametrize("k", [1, 3, 7, 15, 32])
def test_graph_ties_and_duplicates(ccm, k):
    rng = np.random.default_rng(k)
    A = rng.integers(0, 4, size=(120, 3)).astype(np.float64)   # many exact ties
    A[10] = A[11] = A[12]
    _check(ccm, A, k, 0.5)


def test_graph_exact_fallback_path(ccm, monkeypatch):
    """Every row through the exhaustive float64 search gives the same graph."""
    A, _, wl = synth.make_workload("gmm200_d2", 3)
    monkeypatch.setenv("CCM_KNN_FORCE_EXACT", "1")
    _check(ccm, A, wl.k, 0.0)
    rng = np.random.default_rng(5)
    B = rng.integers(0, 3, size=(90, 2)).astype(np.float64)
    _check(ccm, B, 6, 0.5)


def test_graph_tiny_and_edge_cases(ccm):
    A = np.array([[0.0], [1.0]])
    E = _check(ccm, A, 1, 0.5)
    assert E.tolist() == [[0, 1]]
    A = np.random.default_rng(0).normal(size=(65, 5))     # ragged tile (65 rows)
    _check(ccm, A, 32, 0.0)
    with pytest.raises(ccm.CCMError):
        ccm.build_graph(torch.zeros((5, 2), dtype=torch.float64, device="cuda:0"), 5, 0.5)
    bad = torch.tensor([[0.0, np.nan], [1.0, 2.0], [3.0, 1.0]], dtype=torch.float64,
                       device="cuda:0")
    with pytest.raises(ccm.CCMError):
        ccm.build_graph(bad, 1, 0.5)
    with pytest.raises(ccm.CCMError):   # all points equal: median distance 0
        ccm.build_graph(torch.zeros((6, 2), dtype=torch.float64, device="cuda:0"), 2, 0.0)


def test_graph_full_mnist_shape_sampled_rows(ccm):
    """Full n = 10,000, d = 784: sampled rows against the oracle one by one."""
    A, _, wl = synth.make_workload("mnist10k_d784", 0)
    E, w, ph = _gpu_graph(ccm, A, wl.k, 0.0)
    n = A.shape[0]
    assert n * wl.k / 2 <= E.shape[0] <= n * wl.k
    adj = [[] for _ in range(n)]
    for a, b in E:
        adj[a].append(b)
        adj[b].append(a)
    rng = np.random.default_rng(0)
    rows = rng.choice(n, 24, replace=False)
    Nr = ograph.knn_rows(A, wl.k, rows)
    for r, i in enumerate(rows):
        assert set(Nr[r]) <= set(adj[i])
        extra = sorted(set(adj[i]) - set(Nr[r]))
        if extra:
            Ne = ograph.knn_rows(A, wl.k, np.array(extra))
            for t, j in enumerate(extra):
                assert i in Ne[t]
    # weights of sampled edges against the oracle's formula with the GPU's phi
    sel = rng.choice(E.shape[0], 200, replace=False)
    D = ograph.edge_sqdist(A, E[sel])
    np.testing.assert_allclose(w[sel], np.exp(-(ph * D)), rtol=5e-16, atol=1e-300)
    Dall = ograph.edge_sqdist(A, E)
    assert ph == 1.0 / np.sort(Dall)[(Dall.size - 1) // 2]
