"""Gradients of a loss of the clustering path by implicit differentiation (oracle).

Not in the paper. For a loss L = sum_t L_t(X*(gamma_t)) with G_t = dL_t/dX, the
gradient with respect to the data A and the weights w (edges fixed) follows
from the optimality conditions of model CCM (Sec. 1) away from fusion events:

* clusters c: connected components of fused edges (oracle.labels rule);
  Q (n x K) assigns nodes to clusters; M = diag(cluster sizes) (x) I_d;
* N: edges joining two different clusters, with s_l = (x_i - x_j)/||x_i - x_j||
  and c_l = r_l / ||x_i - x_j||, r_l = gamma w_l;
* while the fusion pattern is fixed, the cluster values mu solve
  min_mu 1/2 sum_c sum_{i in c} ||mu_c - a_i||^2 + sum_{l in N} r_l ||mu_c(i) - mu_c(j)||,
  whose Hessian is H = M + sum_{l in N} c_l (e_c(i) - e_c(j))(e_c(i) - e_c(j))^T (x) (I - s_l s_l^T);
* with H lambda = Q^T G:  dL/da_i = lambda_c(i),
  dL/dw_l = -gamma s_l^T (lambda_c(i) - lambda_c(j)) for l in N and 0 for the rest.

The reduced system is assembled densely and solved with numpy.linalg.solve.

Pinned by: the n = 2 closed form and central finite differences of oracle.ssnal
(tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np

from .labels import labels as _labels

__all__ = ["vjp_one", "path_vjp"]


def vjp_one(A, edges, w, gamma, X, G):
    A = np.asarray(A, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.int64)
    n, d = A.shape
    lab = _labels(X, edges)
    K = int(lab.max()) + 1
    ci, cj = lab[edges[:, 0]], lab[edges[:, 1]]
    N = np.nonzero(ci != cj)[0]
    diff = X[edges[N, 0]] - X[edges[N, 1]]
    nd = np.sqrt(np.sum(diff * diff, axis=1))
    s = diff / nd[:, None]
    c = gamma * w[N] / nd
    sizes = np.bincount(lab, minlength=K).astype(np.float64)
    H = np.kron(np.diag(sizes), np.eye(d))
    I = np.eye(d)
    for t, l in enumerate(N):
        a, b = ci[l], cj[l]
        P = c[t] * (I - np.outer(s[t], s[t]))
        sa, sb = slice(a * d, a * d + d), slice(b * d, b * d + d)
        H[sa, sa] += P
        H[sb, sb] += P
        H[sa, sb] -= P
        H[sb, sa] -= P
    QtG = np.zeros((K, d))
    np.add.at(QtG, lab, G)
    lam = np.linalg.solve(H, QtG.reshape(-1)).reshape(K, d)
    dA = lam[lab]
    dw = np.zeros(edges.shape[0])
    dw[N] = -gamma * np.sum(s * (lam[ci[N]] - lam[cj[N]]), axis=1)
    return dA, dw


def path_vjp(A, edges, w, gammas, Xs, Gs):
    dA = np.zeros_like(np.asarray(A, dtype=np.float64))
    dw = np.zeros(np.asarray(edges).shape[0])
    for t, g in enumerate(gammas):
        a, b = vjp_one(A, edges, w, g, Xs[t], Gs[t])
        dA += a
        dw += b
    return dA, dw
