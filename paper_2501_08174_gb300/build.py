"""Build libocgs.so in-tree for sm_103a (GB300) with nvcc.

Every ``csrc/*.cu`` translation unit is compiled in parallel to an object in
``_build/`` and linked into ``paper_2501_08174_gb300/libocgs.so`` (CUDA
runtime linked statically).  Objects are rebuilt only when their source or a
header is newer.  nvcc cross-compiles, so this runs without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libocgs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libocgs")
    return cand


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def _obj_dir(extra: list[str]) -> str:
    """Objects live in a directory named for the extra flags, so a build with other flags
    (a diagnostic build, say) never reuses them."""
    import hashlib
    tag = hashlib.sha256(" ".join(extra).encode()).hexdigest()[:12] if extra else "default"
    return os.path.join(BUILD, tag)


def _compile(src: str, extra: list[str], verbose: bool) -> str:
    obj = os.path.join(_obj_dir(extra), os.path.basename(src)[:-3] + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _headers_mtime()):
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr.strip():
        print(r.stderr, flush=True)
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile and link libocgs.so; return its path."""
    extra = list(extra or [])
    os.makedirs(_obj_dir(extra), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, verbose), srcs))
    # relink when an object is newer or the library was linked from another flag set
    stamp = LIB + ".flags"
    same_flags = os.path.exists(stamp) and open(stamp).read() == " ".join(extra)
    if not os.path.exists(LIB) or not same_flags or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        with open(stamp, "w") as f:
            f.write(" ".join(extra))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
