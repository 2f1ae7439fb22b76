"""Build libccm.so in-tree with nvcc for sm_103a (B300).

Usage: python -m paper_2501_15964_b300.build   (or build() from Python).
Each .cu file is compiled to an object in parallel, then linked into
paper_2501_15964_b300/libccm.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libccm.so")
BUILD = os.path.join(HERE, "_build")
# bounds-checked build: the same sources with CCM_DEBUG_BOUNDS (index checks that
# record the first bad index and skip the access; see ssnal_kernels.cuh)
OUT_DEBUG = os.path.join(HERE, "libccm_debug.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _needs(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    deps.append(os.path.join(HERE, "..", "include", "ccm.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def _compile(src, verbose=False, debug=False):
    obj = os.path.join(BUILD_DEBUG if debug else BUILD, os.path.basename(src)[:-3] + ".o")
    if not _needs(obj, src):
        return obj, ""
    cmd = ["nvcc", *ARCH, *FLAGS, *(["-DCCM_DEBUG_BOUNDS"] if debug else []), "-c", src, "-o", obj]
    if verbose:
        cmd[1:1] = ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj, r.stderr


def build(verbose: bool = False, jobs: int | None = None, debug: bool = False) -> str:
    """Compile every .cu file and link libccm.so (debug=True: the bounds-checked
    libccm_debug.so). Objects are rebuilt only when a source or header changed."""
    out, bdir = (OUT_DEBUG, BUILD_DEBUG) if debug else (OUT, BUILD)
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, debug), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    if (not os.path.exists(out)) or any(os.path.getmtime(o) > os.path.getmtime(out) for o in objs):
        cmd = ["nvcc", *ARCH, "-shared", "-o", out, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
