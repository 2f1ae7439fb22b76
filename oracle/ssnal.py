"""Model CCM (q = 2, 1 or inf) along a gamma path by a textbook SSNAL (oracle).

Sec. 1 states the model and names SSNAL (semismooth Newton augmented
Lagrangian) as the second-order solver; the paper prints none of its steps.
The steps below are restated from convex analysis:

Split z_l = (BX)_l with p(Z) = sum_l r_l ||z_l||, r_l = gamma w_l. The augmented
Lagrangian with multiplier U and penalty sigma, minimised over Z, leaves
    phi(X) = 1/2||X - A||^2 + (1/sigma) sum_l h_l(y_l) - ||U||^2 / (2 sigma),
    y = U + sigma B X,  h_l(y) = ||y||^2/2 if ||y|| <= r_l else r_l||y|| - r_l^2/2,
which is convex and C^1 with
    grad phi(X) = X - A + B^T Pi(y),   Pi = row-wise projection onto ||u_l|| <= r_l.
One outer step: X <- argmin phi (semismooth Newton: solve V D = -grad phi with
V = I + sigma B^T P B, P_l = I if ||y_l|| <= r_l, else (r_l/||y_l||)(I - yhat yhat^T),
P_l = 0 when r_l = 0; Armijo backtracking on phi), then U <- Pi(U + sigma B X).
The gamma path is solved in increasing order, warm-started from the previous
(X, U, sigma); U stays feasible because r grows with gamma.

The minimiser X* is unique (model CCM is strongly convex), so this oracle is
compared with the GPU path on X only; U is not unique when the graph has cycles.

Pinned by: the n = 2 closed form, gamma = 0, the exact 1-D path
(oracle.exact1d), the tree-graph fusion threshold, large-gamma centroids,
invariances, and agreement with the independent ADMM solver
(tests/test_oracle_solvers.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .kkt import incidence, kkt, proj_l1ball

__all__ = ["solve", "solve_path"]


def _eval(X, A, U, B, r, sigma, q=2):
    """phi (without its X-independent term), grad phi, Pi(y), y, ||y_l||.

    For q = 1 the ball is ||u_l||_inf <= r_l: Pi clamps each element to
    [-r_l, r_l], h is the elementwise Huber function, and the last return is |y|.
    For q = inf the ball is ||u_l||_1 <= r_l, Pi is the l1-ball projection,
    h(y) = (||y||^2 - ||y - Pi(y)||^2) / 2 (the Moreau envelope identity that also
    gives the q = 2 and q = 1 forms), and the last return is Pi(y).
    """
    Y = U + sigma * (B @ X)
    if q == np.inf:
        PiY = proj_l1ball(Y, r)
        D = Y - PiY
        h = 0.5 * (np.sum(Y * Y, axis=1) - np.sum(D * D, axis=1))
        phi = 0.5 * np.sum((X - A) ** 2) + np.sum(h) / sigma
        G = X - A + B.T @ PiY
        return phi, G, PiY, Y, PiY
    if q == 1:
        ay = np.abs(Y)
        rr = r[:, None]
        hin = ay <= rr
        h = np.where(hin, 0.5 * Y * Y, rr * ay - 0.5 * rr * rr)
        phi = 0.5 * np.sum((X - A) ** 2) + np.sum(h) / sigma
        PiY = np.clip(Y, -rr, rr)
        G = X - A + B.T @ PiY
        return phi, G, PiY, Y, ay
    ny = np.sqrt(np.sum(Y * Y, axis=1))
    inside = ny <= r
    h = np.where(inside, 0.5 * ny * ny, r * ny - 0.5 * r * r)
    phi = 0.5 * np.sum((X - A) ** 2) + np.sum(h) / sigma
    scale = np.ones_like(ny)
    out = ~inside
    scale[out] = r[out] / ny[out]
    PiY = Y * scale[:, None]
    G = X - A + B.T @ PiY
    return phi, G, PiY, Y, ny


def _mask_l1(ay, r):
    """q = 1: P_l = diag(mask_l), mask = 1 where |y_k| <= r_l (and r_l > 0)."""
    return ((ay <= r[:, None]) & (r[:, None] > 0)).astype(np.float64)


def _linf_parts(Y, PiY, r):
    """q = inf: P_l = diag(mask_l) - s_l s_l^T (an element of the generalized
    Jacobian of the l1-ball projection). Inside rows (||y_l||_1 <= r_l, r_l > 0):
    mask = 1, s = 0 (P = I). Outside rows: mask = 1 on the support S of Pi(y_l)
    and s = sign(y_l) mask / sqrt(|S|). r_l = 0: mask = 0 (P = 0)."""
    m, d = Y.shape
    mask = np.zeros((m, d))
    svec = np.zeros((m, d))
    l1 = np.sum(np.abs(Y), axis=1)
    for l in range(m):
        if r[l] <= 0.0:
            continue
        if l1[l] <= r[l]:
            mask[l] = 1.0
            continue
        S = PiY[l] != 0.0
        mask[l, S] = 1.0
        svec[l, S] = np.sign(Y[l, S]) / np.sqrt(np.count_nonzero(S))
    return mask, svec


def _jacobian_parts(Y, ny, r):
    """alpha_l and yhat_l of P_l = alpha_l (I - yhat yhat^T), or identity rows."""
    inside = (ny <= r) & (r > 0)
    alpha = np.zeros_like(ny)
    yhat = np.zeros_like(Y)
    alpha[inside] = 1.0
    out = (ny > r) & (r > 0)
    alpha[out] = r[out] / ny[out]
    yhat[out] = Y[out] / ny[out, None]
    return alpha, yhat


def _apply_V(Dv, B, alpha, yhat, sigma, mask=None, svec=None):
    BD = B @ Dv
    if svec is not None:
        s = np.sum(svec * BD, axis=1)
        return Dv + sigma * (B.T @ (mask * BD - s[:, None] * svec))
    if mask is not None:
        return Dv + sigma * (B.T @ (mask * BD))
    s = np.sum(yhat * BD, axis=1)
    PBD = alpha[:, None] * (BD - s[:, None] * yhat)
    return Dv + sigma * (B.T @ PBD)


def _dense_V(n, d, edges, alpha, yhat, sigma, mask=None, svec=None):
    V = np.eye(n * d)
    for l in range(edges.shape[0]):
        if svec is not None:
            P = np.diag(mask[l]) - np.outer(svec[l], svec[l])
        elif mask is not None:
            P = np.diag(mask[l])
        elif alpha[l] == 0.0:
            continue
        else:
            P = alpha[l] * (np.eye(d) - np.outer(yhat[l], yhat[l]))
        i, j = edges[l]
        si, sj = slice(i * d, i * d + d), slice(j * d, j * d + d)
        V[si, si] += sigma * P
        V[sj, sj] += sigma * P
        V[si, sj] -= sigma * P
        V[sj, si] -= sigma * P
    return V


def _newton_direction(G, B, edges, alpha, yhat, sigma, n, d, method, cg_rtol, mask=None,
                      svec=None):
    if method == "dense":
        V = _dense_V(n, d, edges, alpha, yhat, sigma, mask, svec)
        return np.linalg.solve(V, -G.reshape(-1)).reshape(n, d), 0
    op = spla.LinearOperator(
        (n * d, n * d),
        matvec=lambda v: _apply_V(v.reshape(n, d), B, alpha, yhat, sigma, mask,
                                  svec).reshape(-1),
        dtype=np.float64)
    it = [0]

    def cb(_):
        it[0] += 1

    sol, _info = spla.cg(op, -G.reshape(-1), rtol=cg_rtol, atol=0.0,
                         maxiter=20 * n * d, callback=cb)
    return sol.reshape(n, d), it[0]


def solve(A, edges, w, gamma, X0=None, U0=None, sigma0=1.0, tol=1e-11,
          max_outer=300, max_newton=60, method=None, sigma_max=1e4, q=2):
    """Solve model CCM (q = 2, 1 or inf) at one gamma. Returns (X, U, sigma, info)."""
    A = np.asarray(A, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.int64)
    n, d = A.shape
    m = edges.shape[0]
    B = incidence(edges, n)
    r = gamma * np.asarray(w, dtype=np.float64)
    X = A.copy() if X0 is None else np.array(X0, dtype=np.float64)
    U = np.zeros((m, d)) if U0 is None else np.array(U0, dtype=np.float64)
    sigma = float(sigma0)
    if method is None:
        method = "dense" if n * d <= 1200 else "cg"
    nA = np.linalg.norm(A)
    info = dict(outer=0, newton=0, cg=0, ls=0)
    last_kkt = 1.0
    last_etap = None
    res = kkt(A, edges, w, gamma, X, U, q)
    if res["kkt"] <= tol and res["gap"] <= tol:
        info.update(res)
        return X, U, sigma, info
    for outer in range(max_outer):
        eps_in = max(0.5 * tol, 0.1 * last_kkt)
        phi, G, PiY, Y, ny = _eval(X, A, U, B, r, sigma, q)
        for _ in range(max_newton):
            if np.linalg.norm(G) / (1.0 + nA) <= eps_in:
                break
            mask = svec = None
            if q == 1:
                mask = _mask_l1(ny, r)
                alpha = yhat = None
            elif q == np.inf:
                mask, svec = _linf_parts(Y, ny, r)
                alpha = yhat = None
            else:
                alpha, yhat = _jacobian_parts(Y, ny, r)
            gn = np.linalg.norm(G)
            cg_rtol = max(1e-14, min(1e-3, 1e-2 * gn / (1.0 + nA)))
            Dv, cgit = _newton_direction(G, B, edges, alpha, yhat, sigma, n, d, method,
                                         cg_rtol, mask, svec)
            info["cg"] += cgit
            gd = float(np.sum(G * Dv))
            t = 1.0
            slack = 1e-14 * (1.0 + abs(phi))
            while True:
                Xt = X + t * Dv
                phit, Gt, PiYt, Yt, nyt = _eval(Xt, A, U, B, r, sigma, q)
                info["ls"] += 1
                if phit <= phi + 1e-4 * t * gd + slack or t < 1e-10:
                    break
                t *= 0.5
            X, phi, G, PiY, Y, ny = Xt, phit, Gt, PiYt, Yt, nyt
            info["newton"] += 1
            if t < 1e-10:       # no descent left at working precision
                break
        U = PiY
        info["outer"] += 1
        res = kkt(A, edges, w, gamma, X, U, q)
        if res["kkt"] <= tol and res["gap"] <= tol:
            break
        if last_etap is not None and res["eta_p"] > 0.2 * last_etap:
            sigma = min(sigma * 3.0, sigma_max)
        last_etap = res["eta_p"]
        last_kkt = res["kkt"]
    info.update(res)
    info["sigma"] = sigma
    return X, U, sigma, info


def solve_path(A, edges, w, gammas, tol=1e-11, sigma0=1.0, method=None, **kw):
    """Warm-started path over non-decreasing gammas.

    Returns (Xs (T x n x d), Us (T x m x d), infos).
    """
    gammas = np.asarray(gammas, dtype=np.float64)
    if np.any(np.diff(gammas) < 0) or np.any(gammas < 0):
        raise ValueError("gammas must be non-negative and non-decreasing")
    X = U = None
    sigma = sigma0
    Xs, Us, infos = [], [], []
    for g in gammas:
        X, U, sigma, info = solve(A, edges, w, g, X, U, sigma, tol=tol, method=method, **kw)
        Xs.append(X.copy())
        Us.append(U.copy())
        infos.append(info)
    return np.stack(Xs), np.stack(Us), infos
