"""The C ABI library loads and exports every function include/ccm.h declares
(no compute calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ccm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2501_15964_b300 as ccm
    from paper_2501_15964_b300 import build as b
    if not os.path.exists(ccm.lib_path()):
        b.build()
    return ccm.load_library()


def test_header_declares_entry_points():
    names = _declared()
    for want in ["ccm_build_graph", "ccm_solve_path", "ccm_path_vjp", "ccm_labels",
                 "ccm_solve_path_batched", "ccm_create", "ccm_destroy", "ccm_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2501_15964_b300 as ccm
    out = subprocess.run(["nm", "-D", "--defined-only", ccm.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ccm_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_host_side_calls_without_gpu(lib):
    import ctypes as C
    from paper_2501_15964_b300._lib import Options
    o = Options()
    lib.ccm_default_options(C.byref(o))
    assert o.max_outer > 0 and o.sigma0 > 0 and o.precision in (0, 1)
    assert lib.ccm_max_dim() >= 784
    assert isinstance(lib.ccm_last_error(), bytes)
    # invalid arguments are rejected before any device work
    h = C.c_void_p()
    assert lib.ccm_create(None, 0) == 1


def test_package_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2501_15964_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_binding_constants_match_header():
    """The Python binding's q = inf code and the option defaults agree with the
    C header (sigma_max <= 0 selects the per-q penalty cap)."""
    import ctypes as C
    from paper_2501_15964_b300._lib import Q_INF, Options
    from paper_2501_15964_b300.api import _q_arg
    src = open(HEADER).read()
    m = re.search(r"#define\s+CCM_Q_INF\s+(\d+)", src)
    assert m and int(m.group(1)) == Q_INF == 2 ** 31 - 1
    assert _q_arg("inf") == _q_arg(float("inf")) == Q_INF and _q_arg(1) == 1
    import paper_2501_15964_b300 as ccm
    o = Options()
    ccm.load_library().ccm_default_options(C.byref(o))
    assert o.sigma_max <= 0.0 and o.sigma0 == 1.0


def test_bounds_checked_library_exports_every_declared_symbol(lib):
    """The CCM_DEBUG_BOUNDS build (libccm_debug.so) is the same ABI."""
    from paper_2501_15964_b300 import build as b
    from paper_2501_15964_b300._lib import debug_lib_path
    path = debug_lib_path()
    if not os.path.exists(path):
        b.build(debug=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (ccm_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
