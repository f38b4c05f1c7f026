"""Build the CUDA library libgf2x_gb300.so in-tree, for sm_103a only.

Each .cu under csrc/ is compiled in parallel with nvcc, then linked into
``paper_1803_11301_gb300/_build/libgf2x_gb300.so``.  Usage:
``python -m paper_1803_11301_gb300.build`` (or ``__graft_entry__.build()``).
"""

from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB_NAME = "libgf2x_gb300.so"
LIB = os.path.join(OUT, LIB_NAME)
# The same library built with GF2X_DEBUG_BOUNDS (the kernels range-check their
# main global indices and count what falls outside, see include/gf2x.h).
OUT_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, LIB_NAME)
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-fvisibility=hidden", "--expt-relaxed-constexpr",
              "-I", INCLUDE]
# The persistent batch kernel reads data that other blocks of the same launch
# wrote: its global loads are cached in L2 only.
PER_FILE_FLAGS = {"persist.cu": ["-Xptxas", "-dlcm=cg"]}


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgf2x_gb300.so")
    return path


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          debug_bounds: bool = False) -> str:
    """Compile every CUDA source and link the shared library; return its path.
    debug_bounds: the GF2X_DEBUG_BOUNDS library, in its own directory."""
    out, lib = (OUT_DEBUG, LIB_DEBUG) if debug_bounds else (OUT, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + list(extra_flags or []) + (["-DGF2X_DEBUG_BOUNDS"] if debug_bounds else [])
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [cc, *ARCH, *flags, *PER_FILE_FLAGS.get(os.path.basename(src), []), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + f".tmp{os.getpid()}"
    link = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    subprocess.run(link, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
