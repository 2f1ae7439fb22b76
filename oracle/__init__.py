"""CPU oracle for the convex clustering path (test infrastructure only).

Plain, slow, float64 numpy/scipy code that states what the GPU path must
compute, written from the paper's definitions:

* ``graph``   canonical squared distances, exact kNN, symmetrized edge set and
              Gaussian weights (the weights w_ij of the CCM model, Sec. 1 and
              Sec. 2.2 item 1, Data Processor);
* ``ssnal``   the CCM minimiser along a gamma path (model CCM, Sec. 1) by a
              textbook semismooth-Newton augmented Lagrangian method (Sec. 1
              names SSNAL; its steps are restated here from convex analysis);
* ``admm``    an independent second solver (ADMM, Sec. 1 and Table 3) used as a
              cross-check;
* ``kkt``     KKT residuals, primal/dual objectives and the relative duality
              gap of Sec. 4;
* ``labels``  cluster assignment x_i = x_j (Sec. 1) with an absolute 1e-6
              distance threshold;
* ``adjoint`` gradients of a loss of X*(gamma) with respect to A and w by
              implicit differentiation;
* ``exact1d`` exact solutions in 1-D (complete graph, unit weights) used only
              to pin the solvers.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The library in
``paper_2501_15964_b300`` never imports it, and this package never imports the
library: the two share no code. Parity status of each function is stated in its
docstring ("pinned by ..." or "parity unpinned").
"""
from . import graph, kkt, labels, ssnal, admm, adjoint, exact1d  # noqa: F401
