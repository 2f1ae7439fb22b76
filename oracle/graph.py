"""Weighted kNN graph of the CCM model (oracle).

The paper fixes only that w_ij = w_ji >= 0 depend on the data (Sec. 1, after
model CCM) and that the Data Processor computes them (Sec. 2.2 item 1). The
readings used here:

* distance: the canonical squared Euclidean distance
  D_ij = sum_k (a_ik - a_jk)^2 evaluated in binary64 with round-to-nearest, one
  rounding per subtraction, product and addition, features in ascending order,
  no fused multiply-add. D_ij and D_ji are bitwise equal.
* neighbours: for each i, the k points j != i with the smallest (D_ij, j) in
  lexicographic order (ties go to the smaller index; duplicates count).
* edges: the union of the directed kNN pairs, stored once as (min, max) and
  sorted lexicographically; the row index is the edge id.
* weights: w_l = exp(-phi * D_l); phi is given, or 1 / (lower median of the
  edge distances), the lower median being element floor((m-1)/2) of the
  sorted D_l.

Pinned by: brute-force agreement with scikit-learn's exact neighbour search
away from ties, hand-made tie fixtures under tests/golden, and counting
invariants (tests/test_oracle_graph.py).
"""
from __future__ import annotations

import numpy as np

__all__ = ["canonical_sqdist_rows", "knn", "knn_rows", "symmetrize", "edge_sqdist",
           "weights", "build_graph"]


def canonical_sqdist_rows(A: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """D[r, j] for the given rows r and every j, canonical order (see module doc)."""
    A = np.asarray(A, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    acc = np.zeros((rows.size, A.shape[0]), dtype=np.float64)
    for f in range(A.shape[1]):
        delta = A[rows, f][:, None] - A[None, :, f]
        acc = acc + delta * delta
    return acc


def knn_rows(A: np.ndarray, k: int, rows: np.ndarray) -> np.ndarray:
    """Exact k nearest neighbours of the given rows, ties by smaller index."""
    n = A.shape[0]
    if not (0 < k < n):
        raise ValueError("need 0 < k < n")
    D = canonical_sqdist_rows(A, rows)
    D[np.arange(rows.size), rows] = np.inf          # exclude self
    order = np.argsort(D, axis=1, kind="stable")    # stable: equal D keep index order
    return order[:, :k].astype(np.int64)


def knn(A: np.ndarray, k: int, block: int = 256) -> np.ndarray:
    """Exact kNN for every row (n x k, int64)."""
    n = A.shape[0]
    out = np.empty((n, k), dtype=np.int64)
    for s in range(0, n, block):
        rows = np.arange(s, min(n, s + block))
        out[rows] = knn_rows(A, k, rows)
    return out


def symmetrize(nbrs: np.ndarray) -> np.ndarray:
    """Union of directed pairs (i, nbrs[i, :]) as sorted unique (min, max) rows."""
    n, k = nbrs.shape
    i = np.repeat(np.arange(n, dtype=np.int64), k)
    j = nbrs.reshape(-1).astype(np.int64)
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    key = np.unique(lo * n + hi)
    return np.stack([key // n, key % n], axis=1).astype(np.int64)


def edge_sqdist(A: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """Canonical D for each edge (same rounding order as canonical_sqdist_rows)."""
    A = np.asarray(A, dtype=np.float64)
    i, j = edges[:, 0], edges[:, 1]
    acc = np.zeros(edges.shape[0], dtype=np.float64)
    for f in range(A.shape[1]):
        delta = A[i, f] - A[j, f]
        acc = acc + delta * delta
    return acc


def weights(D: np.ndarray, phi: float):
    """Gaussian weights w = exp(-phi * D); phi <= 0 selects 1 / lower median."""
    D = np.asarray(D, dtype=np.float64)
    if phi <= 0:
        med = np.sort(D)[(D.size - 1) // 2]
        if not med > 0:
            raise ValueError("lower median of edge distances is zero")
        phi = 1.0 / med
    return np.exp(-(phi * D)), float(phi)


def build_graph(A: np.ndarray, k: int, phi: float):
    """Edges (m x 2 int64, sorted), weights (m,), phi used."""
    nbrs = knn(A, k)
    edges = symmetrize(nbrs)
    D = edge_sqdist(A, edges)
    w, phi_used = weights(D, phi)
    return edges, w, phi_used
