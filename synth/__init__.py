"""Seeded synthetic inputs for the convex-clustering path.

This module only draws random numbers and names the workloads. It holds none of
the method's arithmetic (no distances, no weights, no solver), so both the CPU
oracle and the CUDA path can take their inputs from here without sharing any
computation.

The paper measures on LIBRAS, COIL-20, LUNG and MNIST (Sec. 3, Table 2); those
datasets are not available here. The generators below stand in for them with
Gaussian mixtures of the same kind of shape (the MNIST-shaped one keeps
n=10,000, d=784, K=10 and values in [0, 1]).

Every generator takes a seed and uses ``numpy.random.default_rng(seed)``; the
order of the draws is fixed by the code below, so the same seed always gives
the same bytes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "gaussian_mixture",
    "mnist_like",
    "make_workload",
    "batched_problems",
    "adjoint_target",
    "gamma_grid",
]


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: data recipe plus graph and path settings."""

    name: str
    n: int
    d: int
    k: int
    phi: float  # > 0: used as given; <= 0: phi = 1 / (lower median of edge distances)
    gamma_lo: float
    gamma_hi: float
    n_gamma: int
    recipe: str
    params: dict = field(default_factory=dict)


def gamma_grid(lo: float, hi: float, count: int) -> np.ndarray:
    """Log-spaced, strictly increasing gamma values (the path of Sec. 1)."""
    return np.logspace(np.log10(lo), np.log10(hi), count)


def gaussian_mixture(rng, n, d, n_comp, center_scale, std_lo, std_hi,
                     sizes="equal", center_dist="normal"):
    """Isotropic Gaussian mixture.

    center_dist "uniform": centers U[-center_scale, center_scale]^d,
    "normal": centers N(0, center_scale^2 I). Per-component std U[std_lo, std_hi]
    (a single value when std_lo == std_hi). sizes "equal": i.i.d. uniform
    component choice; "dirichlet": component probabilities ~ Dirichlet(1) then
    i.i.d. choice. Returns (A, component index).
    """
    if center_dist == "uniform":
        centers = rng.uniform(-center_scale, center_scale, size=(n_comp, d))
    else:
        centers = rng.normal(0.0, center_scale, size=(n_comp, d))
    if std_lo == std_hi:
        stds = np.full(n_comp, float(std_lo))
    else:
        stds = rng.uniform(std_lo, std_hi, size=n_comp)
    if sizes == "dirichlet":
        probs = rng.dirichlet(np.ones(n_comp))
    else:
        probs = np.full(n_comp, 1.0 / n_comp)
    comp = rng.choice(n_comp, size=n, p=probs)
    A = centers[comp] + stds[comp, None] * rng.standard_normal((n, d))
    return np.ascontiguousarray(A, dtype=np.float64), comp.astype(np.int32)


def mnist_like(rng, n=10000, d=784, n_proto=10, zero_prob=0.8, noise=0.05):
    """MNIST-shaped stand-in: sparse prototypes in [0,1]^d plus clipped noise.

    Prototypes U[0,1]^d with each entry zeroed with probability zero_prob;
    n/n_proto points per prototype, shuffled; N(0, noise^2) added; clipped to
    [0, 1].
    """
    proto = rng.uniform(0.0, 1.0, size=(n_proto, d))
    proto[rng.uniform(size=(n_proto, d)) < zero_prob] = 0.0
    comp = np.repeat(np.arange(n_proto), n // n_proto)
    comp = comp[rng.permutation(comp.size)]
    A = proto[comp] + rng.normal(0.0, noise, size=(comp.size, d))
    np.clip(A, 0.0, 1.0, out=A)
    return np.ascontiguousarray(A, dtype=np.float64), comp.astype(np.int32)


WORKLOADS = {
    # n=200 points in 2-D, 4 components, kNN k=10, phi=0.5, 20 gammas
    "gmm200_d2": Workload("gmm200_d2", 200, 2, 10, 0.5, 1e-2, 10.0, 20, "gmm",
                          dict(n_comp=4, center_scale=5.0, std_lo=0.5, std_hi=0.5,
                               sizes="equal", center_dist="uniform")),
    # MNIST-shaped: n=10,000, d=784, k=10, phi = 1/median, 50 gammas
    "mnist10k_d784": Workload("mnist10k_d784", 10000, 784, 10, 0.0, 1e-3, 1e2, 50, "mnist"),
    # n=200,000, d=50, 100 components, k=10, phi=0.5 as stated, 30 gammas
    "gmm200k_d50": Workload("gmm200k_d50", 200000, 50, 10, 0.5, 1e-3, 1e2, 30, "gmm",
                            dict(n_comp=100, center_scale=5.0, std_lo=0.5, std_hi=1.5,
                                 sizes="dirichlet", center_dist="normal")),
    # same data with phi = 1/median (the phi=0.5 variant barely fuses)
    "gmm200k_d50_medphi": Workload("gmm200k_d50_medphi", 200000, 50, 10, 0.0, 1e-3, 1e2, 30,
                                   "gmm", dict(n_comp=100, center_scale=5.0, std_lo=0.5,
                                               std_hi=1.5, sizes="dirichlet",
                                               center_dist="normal")),
    # adjoint workload: n=20,000, d=64, 20 components N(0,16 I), std 1, 10 gammas
    "gmm20k_d64": Workload("gmm20k_d64", 20000, 64, 10, 0.0, 1e-2, 10.0, 10, "gmm",
                           dict(n_comp=20, center_scale=4.0, std_lo=1.0, std_hi=1.0,
                                sizes="equal", center_dist="normal")),
}


def make_workload(name: str, seed: int = 0, n: int | None = None):
    """Draw the data matrix A (n x d, float64) for a named workload.

    ``n`` overrides the point count (same recipe, smaller sample) for tests.
    Returns (A, components, workload).
    """
    wl = WORKLOADS[name]
    rng = np.random.default_rng(seed)
    nn = wl.n if n is None else int(n)
    if wl.recipe == "mnist":
        n_proto = 10
        nn = (nn // n_proto) * n_proto
        A, comp = mnist_like(rng, n=nn, d=wl.d, n_proto=n_proto)
    else:
        p = wl.params
        A, comp = gaussian_mixture(rng, nn, wl.d, p["n_comp"], p["center_scale"],
                                   p["std_lo"], p["std_hi"], p["sizes"], p["center_dist"])
    return A, comp, wl


def batched_problems(seed: int = 0, count: int = 256, n_lo: int = 500, n_hi: int = 5000,
                     d: int = 16):
    """Many independent small problems of uneven size (the batched form).

    Each problem: n ~ U{n_lo..n_hi}, K ~ U{2..20} components with centers
    N(0, 25 I) and per-component std U[0.5, 1.5]; k ~ U{5..15}; phi = 1/median;
    25 gammas log-spaced in [1e-3, 1e2]. Returns a list of dicts.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        K = int(rng.integers(2, 21))
        k = int(rng.integers(5, 16))
        A, comp = gaussian_mixture(rng, n, d, K, 5.0, 0.5, 1.5, "equal", "normal")
        out.append(dict(A=A, comp=comp, k=k, phi=0.0,
                        gammas=gamma_grid(1e-3, 1e2, 25)))
    return out


def adjoint_target(seed: int, n: int, d: int) -> np.ndarray:
    """Target T ~ N(0, 1) for the loss sum_t ||X*(gamma_t) - T||_F^2."""
    rng = np.random.default_rng(10_000 + seed)
    return rng.standard_normal((n, d))
