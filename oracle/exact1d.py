"""Exact CCM solutions in one dimension (oracle pin).

For d = 1, the complete graph and w_ij = 1, model CCM (Sec. 1) reads
    min 1/2 sum_i (x_i - a_i)^2 + gamma sum_{i<j} |x_i - x_j|.
If the points are grouped into blocks G_1 < ... < G_K of consecutive sorted
a-values that share one value c_k, the derivative of the objective in c_k is
    sum_{i in G_k} (c_k - a_i) + gamma |G_k| (below_k - above_k),
with below_k / above_k the number of points in lower / higher blocks, so
    c_k = mean(a over G_k) - gamma (below_k - above_k).
The blocks are found by merging adjacent blocks whose values are out of order
(pool adjacent violators), and the result is certified, not assumed: it must be
strictly increasing between blocks, and inside every block each prefix of
sorted members must satisfy
    sum_{prefix} (mean_k - a_i) <= gamma * |prefix| * (|G_k| - |prefix|),
which is the condition for a subgradient of the in-block |x_i - x_j| terms
(each in [-gamma, gamma]) to balance the block. ``solve`` raises if the
certificate fails.

This is independent of the SSNAL and ADMM oracles (no iteration, no linear
algebra) and is used to pin them.
"""
from __future__ import annotations

import numpy as np

__all__ = ["solve", "complete_graph"]


def complete_graph(n: int) -> np.ndarray:
    i, j = np.triu_indices(n, 1)
    return np.stack([i, j], axis=1).astype(np.int64)


def solve(a: np.ndarray, gamma: float) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    n = a.size
    order = np.argsort(a, kind="stable")
    s = a[order]
    blocks = [[k] for k in range(n)]  # indices into s

    def value(b_idx, blist):
        below = sum(len(blist[t]) for t in range(b_idx))
        above = n - below - len(blist[b_idx])
        return float(np.mean(s[blist[b_idx]])) - gamma * (below - above)

    changed = True
    while changed:
        changed = False
        vals = [value(t, blocks) for t in range(len(blocks))]
        for t in range(len(blocks) - 1):
            if vals[t] >= vals[t + 1]:
                blocks[t] = blocks[t] + blocks[t + 1]
                del blocks[t + 1]
                changed = True
                break
    vals = [value(t, blocks) for t in range(len(blocks))]
    # certificate
    for t in range(len(blocks) - 1):
        if not vals[t] < vals[t + 1]:
            raise RuntimeError("1-D certificate failed: blocks out of order")
    for blk in blocks:
        mem = s[blk]
        mu = float(np.mean(mem))
        size = len(blk)
        run = 0.0
        for p in range(1, size):
            run += mu - mem[p - 1]
            if run > gamma * p * (size - p) * (1 + 1e-12) + 1e-12:
                raise RuntimeError("1-D certificate failed: block cannot stay fused")
    x_sorted = np.empty(n)
    for t, blk in enumerate(blocks):
        x_sorted[blk] = vals[t]
    x = np.empty(n)
    x[order] = x_sorted
    return x
