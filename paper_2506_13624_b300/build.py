"""Build the in-tree CUDA library ``libbmpc.so`` for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libbmpc.so")
SOURCES = [os.path.join(CSRC, f) for f in ("bmpc_kernel.cu", "bmpc_api.cu", "bmpc_static.cu", "mlp_kernels.cu",
                                          "tree_lqr.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "bmpc_layout.h"), os.path.join(ROOT, "include", "bmpc.h"),
                  os.path.join(ROOT, "include", "bmpc_mlp.h"), os.path.join(ROOT, "include", "bmpc_lqr.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every source to an object in parallel (each translation unit on its own), then
    links the shared library; skipped while the library is newer than every source and header."""
    stale = not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS)
    if not (force or stale):
        return LIB
    tmp = tempfile.mkdtemp(prefix="bmpc_build_")
    try:
        def compile_one(src):
            obj = os.path.join(tmp, os.path.basename(src) + ".o")
            cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            subprocess.check_call(cmd)
            return obj

        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(compile_one, SOURCES))
        out = LIB + ".tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", out, *objs, "-lcudart"])
        os.replace(out, LIB)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
    print(LIB)
