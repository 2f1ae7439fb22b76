"""Model CCM (q = 2, 1 or inf) by ADMM (oracle cross-check).

ADMM is one of the three solvers the paper's package offers (Sec. 1, Table 1,
Table 3). Here it is a second, independent route to the unique minimiser X*,
used only to pin oracle.ssnal. Splitting z_l = (BX)_l, multiplier U, penalty
sigma:
    X <- (I + sigma L)^{-1} (A + B^T (sigma Z - U)),   L = B^T B (graph Laplacian)
    Z <- prox_{p/sigma}(B X + U / sigma)
    U <- U + sigma (B X - Z)
The X-step uses a sparse LU factorisation of I + sigma L (n x n, applied to each
of the d columns).

Pinned by: agreement with oracle.ssnal and the exact 1-D path.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .kkt import incidence, kkt, prox_group, prox_l1, prox_linf

__all__ = ["solve"]


def solve(A, edges, w, gamma, sigma=1.0, tol=1e-10, max_iter=200000, check_every=50, q=2):
    A = np.asarray(A, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.int64)
    n, d = A.shape
    B = incidence(edges, n)
    r = gamma * np.asarray(w, dtype=np.float64)
    L = (B.T @ B).tocsc()
    solve_x = spla.factorized((sp.identity(n, format="csc") + sigma * L).tocsc())
    X = A.copy()
    Z = B @ X
    U = np.zeros_like(Z)
    res = None
    for it in range(1, max_iter + 1):
        rhs = A + B.T @ (sigma * Z - U)
        X = np.column_stack([solve_x(rhs[:, c]) for c in range(d)])
        BX = B @ X
        prox = prox_l1 if q == 1 else (prox_linf if q == np.inf else prox_group)
        Z = prox(BX + U / sigma, r / sigma)
        U = U + sigma * (BX - Z)
        if it % check_every == 0:
            res = kkt(A, edges, w, gamma, X, U, q)
            if res["kkt"] <= tol and res["gap"] <= tol:
                break
    if res is None:
        res = kkt(A, edges, w, gamma, X, U, q)
    res["iters"] = it
    return X, U, res
