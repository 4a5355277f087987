"""Builds libgh.so (the CUDA library behind include/gh.h) in-tree for sm_103a.

Each .cu file under csrc/ is compiled to an object in parallel, then linked
into paper_2307_16550_gb300/lib/libgh.so with the static CUDA runtime. Host
code is compiled with -ffp-contract=off so that float64 expressions evaluate
with the documented rounding on every host architecture.

The library carries the build id of its sources (source_hash(): SHA-256 of
every csrc/*.cu, csrc/*.cuh and include/gh.h, first 16 hex digits), returned
by gh_build_id(); lib/libgh.so.id records it beside the library, and a
library whose id differs from the sources' is rebuilt.

    python -m paper_2307_16550_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libgh.so")
OBJDIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-fvisibility=hidden",
              "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "gh.h")]


def source_hash() -> str:
    """Build id of the library sources (file names and contents)."""
    import hashlib
    h = hashlib.sha256()
    for p in sorted(_deps()):
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _id_path(lib: str) -> str:
    return lib + ".id"


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(_id_path(LIB)):
        return False
    with open(_id_path(LIB)) as f:
        if f.read().strip() != source_hash():
            return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None, out=None) -> str:
    """Compile and link libgh.so if any source is newer; returns its path.

    extra_flags (e.g. ["-DGH_HOP_U=2"]) and out (another library path) build a
    variant of the library, always from scratch, for tuning experiments."""
    lib = out or LIB
    if not force and not extra_flags and out is None and up_to_date():
        return LIB
    objdir = OBJDIR if out is None else out + ".objs"
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    cc = nvcc()
    bid = source_hash()
    flags = list(NVCC_FLAGS) + [f'-DGH_BUILD_ID="{bid}"'] + list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, file=sys.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(_id_path(lib), "w") as f:
        f.write(bid + "\n")
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
