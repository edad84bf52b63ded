"""Build the CUDA library ``libcflr.so`` in-tree for sm_103a (nvcc, no cmake).

Each translation unit compiles in its own nvcc process (in parallel), then
nvcc links the shared library.  Rebuilds only when a source is newer than
the library.  ``libcflr_checked.so`` is the same library compiled with
CFLR_CHECKED: indices that come from data are tested before use, and a failed
test ends the solve with CFLR_ECUDA instead of an out-of-bounds access (the
binding loads it when CFLR_LIBRARY=checked).
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libcflr.so")
LIB_CHECKED = os.path.join(HERE, "libcflr_checked.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "cflr.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build both libraries (each only when stale); returns the normal one."""
    libs = [(LIB, []), (LIB_CHECKED, ["-DCFLR_CHECKED"])]
    todo = [(lib, extra) for lib, extra in libs if force or _stale(lib)]
    if not todo:
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = {lib: [] for lib, _ in todo}
    cmds = []
    for lib, extra in todo:
        tag = "checked." if extra else ""
        for src in sources():
            obj = os.path.join(BUILD_DIR, tag + os.path.basename(src) + ".o")
            objs[lib].append(obj)
            lang = ["-x", "cu"] if src.endswith(".cu") else []
            cmds.append([nvcc] + ARCH + FLAGS + extra + lang + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
    with ThreadPoolExecutor(max_workers=max(1, len(cmds))) as ex:
        list(ex.map(run, cmds))
    for lib, _ in todo:
        tmp = lib + ".%d.tmp" % os.getpid()
        run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs[lib] + ["-lcudart"])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
