"""ccm_labels_noalloc: the allocation-free labels entry point.

Callers that cannot allocate device memory (inside a pool or allocator that
forbids cudaMalloc/cudaFree, or with device memory fully reserved up front) get
labels from a fixed static scratch array instead of a context. This test calls
it through the C ABI twice in a row and checks both results against
ccm_labels; labels are integers, so the comparison is exact. It sits in its own
file, collected last, and passes alone in a fresh process or after the others.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import graph as ograph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    import paper_2501_15964_b300 as ccm
    lib = ccm.load_library()
    fn = lib.ccm_labels_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                   C.POINTER(C.c_int32), C.c_void_p]
    return ccm, lib, fn


def _case(seed, n, d, k, gamma):
    ccm, _, _ = _lib()
    A, _, _ = synth.make_workload("gmm20k_d64", seed, n=n)
    A = A[:, :d].copy()
    E, w, _ = ograph.build_graph(A, k, 0.0)
    At = torch.tensor(A, device="cuda:0")
    Et = torch.tensor(E, dtype=torch.int32, device="cuda:0")
    wt = torch.tensor(w, device="cuda:0")
    X, L, _, _ = ccm.solve_path(At, Et, wt, [gamma], tol=2e-7)
    return X[0].contiguous(), Et, L[0]


@pytest.mark.parametrize("seed,n,d,k,gamma", [(0, 3000, 16, 8, 0.5), (1, 700, 64, 10, 2.0)])
def test_noalloc_labels_match_ccm_labels_twice(seed, n, d, k, gamma):
    ccm, lib, fn = _lib()
    X, Et, L_path = _case(seed, n, d, k, gamma)
    L_ref, K_ref = ccm.labels(X, Et)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):                       # the static scratch is reused
        out = torch.full((n,), -7, dtype=torch.int32, device="cuda:0")
        K = C.c_int32(-1)
        st = fn(C.c_void_p(X.data_ptr()), n, d, C.c_void_p(Et.data_ptr()), Et.shape[0],
                C.c_void_p(out.data_ptr()), C.byref(K), stream)
        assert st == 0, lib.ccm_last_error().decode()
        torch.cuda.synchronize()
        assert torch.equal(out, L_ref)
        assert torch.equal(out, L_path)
        assert K.value == K_ref


def test_noalloc_rejects_oversize():
    ccm, lib, fn = _lib()
    X = torch.zeros((4, 2), dtype=torch.float64, device="cuda:0")
    E = torch.tensor([[0, 1]], dtype=torch.int32, device="cuda:0")
    out = torch.empty(4, dtype=torch.int32, device="cuda:0")
    K = C.c_int32(0)
    st = fn(C.c_void_p(X.data_ptr()), (1 << 18) + 1, 2, C.c_void_p(E.data_ptr()), 1,
            C.c_void_p(out.data_ptr()), C.byref(K), None)
    assert st == 1
    assert "maximum" in lib.ccm_last_error().decode()
