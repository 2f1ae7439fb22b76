"""Convex clustering (model CCM; q = 2, 1 or inf) along a gamma path on one B300.

Thin Python binding of ``libccm.so`` (C ABI declared in ``include/ccm.h``).
Every computation runs in the library's CUDA kernels; this module only
marshals arguments. PyTorch provides device memory and streams.

There is no CPU fallback: importing works without a GPU (so the build can be
checked), but every call needs the compiled library and a CUDA device and
raises otherwise.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    CCMError,
    Context,
    Options,
    PREC_FP64,
    Q_INF,
    PREC_MIXED,
    ENGINE_AUTO,
    ENGINE_BLOCK,
    ENGINE_GRID,
    lib_path,
    load_library,
    exported_symbols,
)
from .api import (  # noqa: F401
    build_graph,
    solve_path,
    labels,
    path_vjp,
    solve_path_batched,
    solve_path_admm,
    solve_path_ama,
    last_profile,
    last_graph_info,
    launch_count,
    CCMPath,
    default_context,
)
