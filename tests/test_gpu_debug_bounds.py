"""The bounds-checked build (libccm_debug.so, compiled with CCM_DEBUG_BOUNDS).

Its kernels that gather through the CSR incidence records check every record's
edge id and endpoint against the problem's sizes before any memory access; a
bad record is skipped and recorded, and the call returns CCM_ERR_BOUNDS (8)
with a message naming the kernel. Nothing traps.

Each case runs in a fresh process that loads the debug library through
CCM_LIBRARY: (1) a valid grid-engine solve gives the same X as the normal
library; (2) with CCM_DEBUG_CORRUPT set, the engine overwrites one incidence
record's endpoint with n + 3 right after building the CSR (before any kernel
reads it), and the call must fail with CCM_ERR_BOUNDS.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2501_15964_b300 as ccm, synth
from oracle import graph as og
A, _, wl = synth.make_workload("gmm200_d2", 0)
E, w, _ = og.build_graph(A, wl.k, wl.phi)
At = torch.tensor(A, device="cuda:0")
Et = torch.tensor(E, dtype=torch.int32, device="cuda:0")
wt = torch.tensor(w, device="cuda:0")
try:
    X, L, U, st = ccm.solve_path(At, Et, wt, [0.05, 0.5], tol=2e-7, engine=1, precision={prec})
    np.save({out!r}, X.cpu().numpy())
    print("STATUS 0")
except ccm.CCMError as e:
    print("STATUS", e.status, str(e))
"""


def _run(tmp_path, lib, corrupt, prec):
    out = str(tmp_path / f"x_{os.path.basename(lib)}_{corrupt}_{prec}.npy")
    env = dict(os.environ, CCM_LIBRARY=lib)
    if corrupt:
        env["CCM_DEBUG_CORRUPT"] = "1"
    else:
        env.pop("CCM_DEBUG_CORRUPT", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, out=out, prec=prec)],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("STATUS")][-1]
    return line, out


@pytest.mark.parametrize("prec", [1, 0])
def test_bounds_checked_build(tmp_path, prec):
    import numpy as np
    from paper_2501_15964_b300._lib import debug_lib_path, lib_path
    normal = os.path.join(ROOT, "paper_2501_15964_b300", "libccm.so")
    debug = debug_lib_path()
    assert os.path.exists(debug), "build libccm_debug.so first (__graft_entry__.build())"
    s_n, x_n = _run(tmp_path, normal, False, prec)
    s_d, x_d = _run(tmp_path, debug, False, prec)
    assert s_n == "STATUS 0" and s_d == "STATUS 0", (s_n, s_d)
    np.testing.assert_array_equal(np.load(x_n), np.load(x_d))  # the checks change no arithmetic
    s_c, _ = _run(tmp_path, debug, True, prec)
    assert s_c.startswith("STATUS 8") and "k_cg_" in s_c, s_c
