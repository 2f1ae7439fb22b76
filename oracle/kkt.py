"""Optimality measures for model CCM with q = 2, q = 1 or q = inf (oracle).

Notation. For edges l = (i, j), i < j: (BX)_l = x_i - x_j; r_l = gamma * w_l;
p(Z) = sum_l r_l ||z_l||_2. The primal is min_X 1/2||X - A||^2 + p(BX) (model
CCM, Sec. 1). Its Lagrangian dual, for U with ||u_l|| <= r_l, is
f_d(U) = <A, B^T U> - 1/2 ||B^T U||^2 (weak duality: f_d(U) <= f_p(X)).

Readings (the paper gives only the gap of Sec. 4):
* eta_D = ||X - A + B^T U||_F / (1 + ||A||_F)          (stationarity in X)
* eta_P = ||BX - prox_p(BX + U)||_F / (1 + ||A||_F)     (U in the subdifferential
  of p at BX, as a natural residual)
* gap   = |f_p - f_d| / (1 + |f_p| + |f_d|)             (Sec. 4)
* kkt   = max(eta_D, eta_P)

For q = 1 the penalty is p(Z) = sum_l r_l ||z_l||_1, the dual ball is
||u_l||_inf <= r_l and prox_p is the elementwise soft threshold. For q = inf
(passed as numpy.inf) the penalty is sum_l r_l ||z_l||_inf, the dual ball is
||u_l||_1 <= r_l and prox_p = I - (projection onto that ball) by the Moreau
decomposition; the projection follows the sort-and-threshold method of Duchi,
Shalev-Shwartz, Singer and Chandra (ICML 2008).

Pinned by: weak duality (gap >= 0 whenever U is feasible), exact zeros at the
closed-form n = 2 solution and at gamma = 0, and agreement of two independent
solvers (tests/test_oracle_solvers.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["incidence", "prox_group", "prox_l1", "proj_l1ball", "prox_linf", "kkt"]


def incidence(edges: np.ndarray, n: int) -> sp.csr_matrix:
    """B (m x n): row l has +1 at edges[l,0] and -1 at edges[l,1]."""
    m = edges.shape[0]
    rows = np.repeat(np.arange(m), 2)
    cols = edges.reshape(-1)
    vals = np.tile(np.array([1.0, -1.0]), m)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, n))


def prox_group(V: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Row-wise prox of r_l ||.||_2: shrink each row by r_l towards 0."""
    nv = np.sqrt(np.sum(V * V, axis=1))
    scale = np.zeros_like(nv)
    big = nv > r
    scale[big] = 1.0 - r[big] / nv[big]
    return V * scale[:, None]


def prox_l1(V: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Elementwise prox of r_l ||.||_1: soft threshold of row l at r_l."""
    return np.sign(V) * np.maximum(np.abs(V) - r[:, None], 0.0)


def proj_l1ball(V: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Row-wise Euclidean projection of V onto {u : ||u||_1 <= r_l}.

    Rows already inside (||v||_1 <= r_l) are returned unchanged. Otherwise the
    magnitudes are sorted in decreasing order (mu_1 >= mu_2 >= ...), rho is the
    largest j with mu_j > (mu_1 + ... + mu_j - r_l) / j, and the result is the
    soft threshold of the row at theta = (mu_1 + ... + mu_rho - r_l) / rho.
    Pinned by the variational inequality at the ball's vertices and by d = 1
    (tests/test_oracle_solvers.py).
    """
    V = np.asarray(V, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    out = V.copy()
    for l in range(V.shape[0]):
        v = V[l]
        av = np.abs(v)
        if np.sum(av) <= r[l]:
            continue
        if r[l] <= 0.0:
            out[l] = 0.0
            continue
        mu = np.sort(av)[::-1]
        cs = np.cumsum(mu)
        j = np.arange(1, mu.size + 1)
        rho = int(np.nonzero(mu * j > cs - r[l])[0][-1]) + 1
        theta = (cs[rho - 1] - r[l]) / rho
        out[l] = np.sign(v) * np.maximum(av - theta, 0.0)
    return out


def prox_linf(V: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Row-wise prox of r_l ||.||_inf (Moreau: v - projection onto the l1 ball)."""
    return np.asarray(V, dtype=np.float64) - proj_l1ball(V, r)


def kkt(A, edges, w, gamma, X, U, q=2):
    """Residuals and objectives at (X, U); returns a dict."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    B = incidence(np.asarray(edges), n)
    r = gamma * np.asarray(w, dtype=np.float64)
    BX = B @ X
    BtU = B.T @ U
    nA = np.linalg.norm(A)
    eta_d = np.linalg.norm(X - A + BtU) / (1.0 + nA)
    if q == 1:
        eta_p = np.linalg.norm(BX - prox_l1(BX + U, r)) / (1.0 + nA)
        pen = np.sum(r * np.sum(np.abs(BX), axis=1))
        nu = np.max(np.abs(U), axis=1) if U.size else np.zeros(0)
    elif q == np.inf:
        eta_p = np.linalg.norm(BX - prox_linf(BX + U, r)) / (1.0 + nA)
        pen = np.sum(r * np.max(np.abs(BX), axis=1)) if BX.size else 0.0
        nu = np.sum(np.abs(U), axis=1)
    else:
        eta_p = np.linalg.norm(BX - prox_group(BX + U, r)) / (1.0 + nA)
        pen = np.sum(r * np.sqrt(np.sum(BX * BX, axis=1)))
        nu = np.sqrt(np.sum(U * U, axis=1))
    fp = 0.5 * np.sum((X - A) ** 2) + pen
    fd = np.sum(A * BtU) - 0.5 * np.sum(BtU * BtU)
    infeas = float(np.max(np.maximum(nu - r, 0.0))) if nu.size else 0.0
    gap = abs(fp - fd) / (1.0 + abs(fp) + abs(fd))
    return dict(eta_d=float(eta_d), eta_p=float(eta_p), kkt=float(max(eta_d, eta_p)),
                fp=float(fp), fd=float(fd), gap=float(gap), dual_infeas=infeas)
