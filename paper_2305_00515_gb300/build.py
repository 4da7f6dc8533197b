"""Build the sm_103a shared library ``_build/libsobel4.so`` in-tree with nvcc.

Each ``csrc/*.cu`` translation unit is compiled in parallel for
``-gencode arch=compute_103a,code=sm_103a`` and linked into one shared library
that exports the C ABI of ``include/sobel4.h``.  Run as a module
(``python -m paper_2305_00515_gb300.build``) or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libsobel4.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _sources(csrc: str = CSRC):
    return sorted(os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(INCLUDE, "sobel4.h")]


def _compile(src: str, verbose: bool, out_dir: str = BUILD, defines=(), csrc: str = CSRC,
             extra=()) -> str:
    obj = os.path.join(out_dir, os.path.basename(src).replace(".cu", ".o"))
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", csrc, *[f"-D{d}" for d in defines], *extra, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _sources() + _headers())


def build(force: bool = False, verbose: bool = False, out_dir: str = None, defines=(),
          src_dir: str = None, extra_flags=()) -> str:
    """Compile and link; `out_dir`, `defines` (kernel tuning macros such as
    SOBEL4_RG_MIN_CTAS=3) and `src_dir` build a separate copy for tuning sweeps."""
    csrc = src_dir or CSRC
    lib = LIB if out_dir is None else os.path.join(out_dir, "libsobel4.so")
    out_dir = BUILD if out_dir is None else out_dir
    if (not force and out_dir == BUILD and not defines and src_dir is None and not extra_flags
            and up_to_date()):
        return LIB
    os.makedirs(out_dir, exist_ok=True)
    srcs = _sources(csrc)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, out_dir, defines, csrc, extra_flags),
                           srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
