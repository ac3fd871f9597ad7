"""Builds libprobesdf.so (the C ABI + sm_103a kernels) in-tree with nvcc.

Each .cu file compiles to an object in parallel; the objects link into one
shared library under paper_2412_10084_gb300/_build/.  The CUDA runtime is
linked statically, so the library needs only the driver at run time.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libprobesdf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libprobesdf.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


# Files the two render kernels are built from (their code, shared headers, and
# the launch configuration in the C ABI layer).
RENDER_FILES = ("render_fwd.cu", "render_bwd.cu", "render_common.cuh", "sample_eval.cuh",
                "mlp_tc.cuh", "tc_sm100.cuh", "internal.h", "abi.cu", "probesdf.h")


def _inputs_digest(flags, only=None):
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            p = os.path.join(d, f)
            if only is not None and f not in only:
                continue
            if os.path.isfile(p):
                h.update(f.encode())
                with open(p, "rb") as fh:
                    h.update(fh.read())
    # the flags enter without machine paths, so a digest names the same build everywhere
    h.update(" ".join(f.replace(INCLUDE, "<include>").replace(CSRC, "<csrc>")
                      for f in flags).encode())
    return h.hexdigest()


def base_flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-I", CSRC]


def source_digest() -> str:
    """Digest of the kernel sources, headers and default flags (the build stamp)."""
    return _inputs_digest(base_flags())


def render_digest() -> str:
    """Digest of the render kernels' sources and the default flags: profile
    figures of those kernels stay valid while it is unchanged."""
    return _inputs_digest(base_flags(), RENDER_FILES)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    flags = base_flags()
    if verbose:
        flags += ["-Xptxas", "-v"]
    digest = _inputs_digest(flags)
    stamp = os.path.join(BUILD, "libprobesdf.sha256")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *flags, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose:
            sys.stderr.write(res.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
