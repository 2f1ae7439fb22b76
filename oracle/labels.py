"""Cluster labels from a solution X (oracle).

Sec. 1 puts a_i and a_j in the same cluster when x_i* = x_j*. Reading: an edge
(i, j) of the graph is fused when the canonical squared distance
sum_k (x_ik - x_jk)^2 (binary64, features in ascending order, no fused
multiply-add) is <= 1e-12, i.e. ||x_i - x_j||_2 <= 1e-6; clusters are the
connected components of the fused edges; the label of a node is the rank of
its component's smallest node index (0 .. K-1).

Pinned by: gamma = 0 gives singletons for distinct points, large gamma gives
the connected components of the graph, and hand-made fixtures
(tests/test_oracle_labels.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

__all__ = ["FUSE_SQDIST", "fused_mask", "labels"]

FUSE_SQDIST = 1e-12


def fused_mask(X: np.ndarray, edges: np.ndarray) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    i, j = edges[:, 0], edges[:, 1]
    acc = np.zeros(edges.shape[0])
    for f in range(X.shape[1]):
        delta = X[i, f] - X[j, f]
        acc = acc + delta * delta
    return acc <= FUSE_SQDIST


def labels(X: np.ndarray, edges: np.ndarray) -> np.ndarray:
    n = X.shape[0]
    f = fused_mask(X, edges)
    e = edges[f]
    G = sp.coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(n, n))
    _, comp = connected_components(G, directed=False)
    # canonical: order components by their smallest member
    first = np.full(comp.max() + 1, n, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(n))
    rank = np.empty_like(first)
    rank[np.argsort(first, kind="stable")] = np.arange(first.size)
    return rank[comp].astype(np.int32)
