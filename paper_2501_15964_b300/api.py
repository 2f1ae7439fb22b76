"""Torch-facing wrappers of the libccm C ABI (argument marshalling only)."""
from __future__ import annotations

import ctypes as C

import torch

from ._lib import (Q_INF, CCMError, Context, GraphInfo, Options, Problem, Profile, Stats,
                   check, load_library)

_CTX: dict[int, Context] = {}


def default_context(device: int | None = None) -> Context:
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2501_15964_b300 needs a CUDA device (no CPU fallback)")
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _CTX:
        _CTX[dev] = Context(dev)
    return _CTX[dev]


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


def _q_arg(q) -> int:
    """The int32 q of the C ABI: 1, 2, or Q_INF for q = inf (math.inf or "inf")."""
    if isinstance(q, str) and q.lower() in ("inf", "infinity"):
        return Q_INF
    if isinstance(q, float) and q == float("inf"):
        return Q_INF
    return int(q)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def make_options(**kw) -> Options:
    o = Options()
    load_library().ccm_default_options(C.byref(o))
    for k, v in kw.items():
        if k in ("X0", "U0"):
            setattr(o, k, v.data_ptr() if v is not None else None)
        else:
            setattr(o, k, v)
    return o


def build_graph(A: torch.Tensor, k: int, phi: float = 0.0, ctx: Context | None = None):
    """Symmetrized exact kNN graph with Gaussian weights (see ccm_build_graph).

    Returns (edges int32 [m, 2], w float64 [m], phi_used)."""
    A = _dev(A, torch.float64, "A")
    n, d = A.shape
    ctx = ctx or default_context(A.device.index)
    cap = n * k
    edges = torch.empty((cap, 2), dtype=torch.int32, device=A.device)
    w = torch.empty(cap, dtype=torch.float64, device=A.device)
    m = C.c_int64(0)
    ph = C.c_double(0.0)
    check(load_library().ccm_build_graph(ctx.handle, _ptr(A), n, d, int(k), float(phi),
                                          _ptr(edges), _ptr(w), cap, C.byref(m), C.byref(ph),
                                          _stream()))
    return edges[: m.value], w[: m.value], ph.value


def solve_path(A, edges, w, gammas, tol: float = 1e-6, q: int = 2, return_U: bool = False,
               labels_out: bool = True, ctx: Context | None = None, raise_on_cap=False,
               X_out: torch.Tensor | None = None, labels_host: torch.Tensor | None = None,
               **options):
    """X*(gamma_t) for every gamma (see ccm_solve_path).

    X_out / labels_host: optional host tensors (float64 [T,n,d], int32 [T,n];
    pinned memory lets the library copy each gamma's X while the next one solves)
    that receive the outputs instead of new device tensors.

    Returns (X [T,n,d] float64, labels [T,n] int32 or None, U [T,m,d] or None,
    stats: list of dicts)."""
    A = _dev(A, torch.float64, "A")
    edges = _dev(edges, torch.int32, "edges")
    w = _dev(w, torch.float64, "w")
    n, d = A.shape
    m = edges.shape[0]
    g = [float(x) for x in gammas]
    T = len(g)
    ctx = ctx or default_context(A.device.index)
    if X_out is not None:
        if (X_out.device.type != "cpu" or X_out.dtype != torch.float64
                or tuple(X_out.shape) != (T, n, d) or not X_out.is_contiguous()):
            raise ValueError("X_out must be a contiguous float64 CPU tensor of shape (T, n, d)")
        X = X_out
    else:
        X = torch.empty((T, n, d), dtype=torch.float64, device=A.device)
    if labels_host is not None:
        if (labels_host.device.type != "cpu" or labels_host.dtype != torch.int32
                or tuple(labels_host.shape) != (T, n) or not labels_host.is_contiguous()):
            raise ValueError("labels_host must be a contiguous int32 CPU tensor of shape (T, n)")
        lab = labels_host
    else:
        lab = torch.empty((T, n), dtype=torch.int32, device=A.device) if labels_out else None
    U = torch.empty((T, m, d), dtype=torch.float64, device=A.device) if return_U else None
    stats = (Stats * T)()
    garr = (C.c_double * T)(*g)
    opt = make_options(**options)
    st = load_library().ccm_solve_path(ctx.handle, _ptr(A), n, d, _ptr(edges), _ptr(w), m, garr,
                                       T, _q_arg(q), float(tol), C.byref(opt), _ptr(X), _ptr(lab),
                                       _ptr(U), stats, _stream())
    if st != 0 and not (st == 5 and not raise_on_cap):
        check(st)
    return X, lab, U, [s.as_dict() for s in stats]


def solve_path_admm(A, edges, w, gammas, tol: float = 1e-6, q: int = 2, return_U: bool = False,
                    labels_out: bool = True, ctx: Context | None = None, raise_on_cap=False,
                    **options):
    """The path of solve_path by ADMM (see ccm_solve_path_admm); same returns."""
    return _solve_path_with("ccm_solve_path_admm", A, edges, w, gammas, tol, q, return_U,
                            labels_out, ctx, raise_on_cap, options)


def solve_path_ama(A, edges, w, gammas, tol: float = 1e-6, q: int = 2, return_U: bool = False,
                   labels_out: bool = True, ctx: Context | None = None, raise_on_cap=False,
                   **options):
    """The path of solve_path by fast AMA (see ccm_solve_path_ama); same returns."""
    return _solve_path_with("ccm_solve_path_ama", A, edges, w, gammas, tol, q, return_U,
                            labels_out, ctx, raise_on_cap, options)


def _solve_path_with(entry, A, edges, w, gammas, tol, q, return_U, labels_out, ctx, raise_on_cap,
                     options):
    A = _dev(A, torch.float64, "A")
    edges = _dev(edges, torch.int32, "edges")
    w = _dev(w, torch.float64, "w")
    n, d = A.shape
    m = edges.shape[0]
    g = [float(x) for x in gammas]
    T = len(g)
    ctx = ctx or default_context(A.device.index)
    X = torch.empty((T, n, d), dtype=torch.float64, device=A.device)
    lab = torch.empty((T, n), dtype=torch.int32, device=A.device) if labels_out else None
    U = torch.empty((T, m, d), dtype=torch.float64, device=A.device) if return_U else None
    stats = (Stats * T)()
    garr = (C.c_double * T)(*g)
    opt = make_options(**options)
    st = getattr(load_library(), entry)(ctx.handle, _ptr(A), n, d, _ptr(edges), _ptr(w), m, garr,
                                        T, _q_arg(q), float(tol), C.byref(opt), _ptr(X), _ptr(lab),
                                        _ptr(U), stats, _stream())
    if st != 0 and not (st == 5 and not raise_on_cap):
        check(st)
    return X, lab, U, [s.as_dict() for s in stats]


def last_profile(ctx: Context | None = None) -> dict:
    ctx = ctx or default_context()
    p = Profile()
    check(load_library().ccm_last_profile(ctx.handle, C.byref(p)))
    return {"matvec_launches": p.matvec_launches, "matvec_ms_total": p.matvec_ms_total,
            "matvec_bytes_total": p.matvec_bytes_total, "kernel_launches": p.kernel_launches,
            "block_lanes": p.block_lanes, "block_quads": p.block_quads,
            "coarse_steps": p.coarse_steps, "coarse_max_aggregates": p.coarse_max_aggregates}


def last_graph_info(ctx: Context | None = None) -> dict:
    """How the last build_graph on the context found its candidates (see
    ccm_last_graph_info): {"candidates": "tensor" | "simt", "per_row", "rows_exhaustive"}."""
    ctx = ctx or default_context()
    g = GraphInfo()
    check(load_library().ccm_last_graph_info(ctx.handle, C.byref(g)))
    return {"candidates": "tensor" if g.candidates == 1 else "simt", "per_row": g.per_row,
            "rows_exhaustive": g.rows_exhaustive}


def launch_count(ctx: Context | None = None) -> int:
    """Kernels launched through the context since it was created."""
    ctx = ctx or default_context()
    return int(load_library().ccm_launch_count(ctx.handle))


def labels(X, edges, ctx: Context | None = None):
    """Cluster labels of one solution X [n,d] (see ccm_labels). Returns (labels, K)."""
    X = _dev(X, torch.float64, "X")
    edges = _dev(edges, torch.int32, "edges")
    n, d = X.shape
    ctx = ctx or default_context(X.device.index)
    out = torch.empty(n, dtype=torch.int32, device=X.device)
    K = C.c_int32(0)
    check(load_library().ccm_labels(ctx.handle, _ptr(X), n, d, _ptr(edges), edges.shape[0],
                                    _ptr(out), C.byref(K), _stream()))
    return out, K.value


def path_vjp(A, edges, w, gammas, X, dLdX, U=None, ctx: Context | None = None):
    """(dL/dA, dL/dw) of sum_t L_t(X*(gamma_t)) given dL/dX (see ccm_path_vjp)."""
    A = _dev(A, torch.float64, "A")
    edges = _dev(edges, torch.int32, "edges")
    w = _dev(w, torch.float64, "w")
    X = _dev(X, torch.float64, "X")
    G = _dev(dLdX, torch.float64, "dLdX")
    n, d = A.shape
    m = edges.shape[0]
    g = [float(x) for x in gammas]
    T = len(g)
    ctx = ctx or default_context(A.device.index)
    dA = torch.empty_like(A)
    dw = torch.empty_like(w)
    garr = (C.c_double * T)(*g)
    Uc = _dev(U, torch.float64, "U") if U is not None else None
    check(load_library().ccm_path_vjp(ctx.handle, _ptr(A), n, d, _ptr(edges), _ptr(w), m, garr,
                                      T, _ptr(X), _ptr(Uc), _ptr(G), _ptr(dA), _ptr(dw),
                                      _stream()))
    return dA, dw


def solve_path_batched(problems, gammas, tol: float = 1e-6, ctx: Context | None = None,
                       **options):
    """Many independent problems in one persistent launch (see ccm_solve_path_batched).

    problems: list of dicts with CUDA tensors A [n,d] float64, edges [m,2] int32,
    w [m] float64. Returns (list of X [T,n,d], list of labels [T,n], stats [P][T])."""
    P = len(problems)
    g = [float(x) for x in gammas]
    T = len(g)
    d = int(problems[0]["A"].shape[1])
    ctx = ctx or default_context(problems[0]["A"].device.index)
    arr = (Problem * P)()
    keep = []
    Xs, Ls = [], []
    for i, pb in enumerate(problems):
        A = _dev(pb["A"], torch.float64, "A")
        E = _dev(pb["edges"], torch.int32, "edges")
        w = _dev(pb["w"], torch.float64, "w")
        if A.shape[1] != d:
            raise ValueError("all problems of a batch share d")
        X = torch.empty((T,) + tuple(A.shape), dtype=torch.float64, device=A.device)
        L = torch.empty((T, A.shape[0]), dtype=torch.int32, device=A.device)
        keep += [A, E, w]
        Xs.append(X)
        Ls.append(L)
        arr[i] = Problem(A.data_ptr(), E.data_ptr(), w.data_ptr(), A.shape[0], E.shape[0],
                         X.data_ptr(), L.data_ptr())
    stats = (Stats * (P * T))()
    garr = (C.c_double * T)(*g)
    opt = make_options(**options)
    st = load_library().ccm_solve_path_batched(ctx.handle, P, arr, d, garr, T, float(tol),
                                               C.byref(opt), stats, _stream())
    if st not in (0, 5):
        check(st)
    flat = [s.as_dict() for s in stats]
    return Xs, Ls, [flat[i * T:(i + 1) * T] for i in range(P)]


class CCMPath(torch.autograd.Function):
    """X*(gamma_1..T) as a differentiable function of (A, w) for fixed edges.

    forward(A, w, edges, gammas, tol) -> X [T,n,d]; backward uses ccm_path_vjp
    (implicit differentiation at the computed path; fusion pattern held fixed)."""

    @staticmethod
    def forward(ctx, A, w, edges, gammas, tol=1e-6):
        X, _, _, _ = solve_path(A, edges, w, gammas, tol=tol, labels_out=False)
        ctx.save_for_backward(A, w, edges, X)
        ctx.gammas = list(gammas)
        return X

    @staticmethod
    def backward(ctx, gX):
        A, w, edges, X = ctx.saved_tensors
        dA, dw = path_vjp(A, edges, w, ctx.gammas, X, gX.contiguous())
        return dA, dw, None, None, None
