"""Build the CUDA library ``_build/libct_gb300.so`` in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then
linked into one shared library exporting the C ABI of ``include/ct.h``.
Rebuilds only what changed (sources newer than their objects, or any header
newer than every object).
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libct_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]
# The eigen stage flushes FP32 denormals (values below 1.2e-38), so that its
# reciprocal square roots and divisions skip their denormal handling; the
# tensors and every quantity derived from them are zero or far above that
# range (the closed form treats the zero tensor apart).
FILE_FLAGS = {name: ["-ftz=true"] for name in ("ct_k_eig.cu", "ct_k_rhoz_eig.cu", "ct_noalloc.cu")}


def nvcc() -> str:
    cand = shutil.which("nvcc")
    if cand:
        return cand
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    return os.path.join(home, "bin", "nvcc")


def _needs(obj: str, src: str, headers) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or any(os.path.getmtime(h) > t for h in headers)


def build(verbose: bool = False, jobs: int | None = None, extra_flags=(), out_dir: str | None = None,
          csrc: str | None = None) -> str:
    """Compile and link; `out_dir` (default the in-tree _build), `extra_flags`
    and `csrc` (another source tree) allow side-by-side builds of variants."""
    BUILD = out_dir or globals()["BUILD"]
    CSRC = csrc or globals()["CSRC"]
    LIB = os.path.join(BUILD, "libct_gb300.so")
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in sources]
    todo = [(s, o) for s, o in zip(sources, objs) if _needs(o, s, headers)]

    def compile_one(so):
        src, obj = so
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *FILE_FLAGS.get(os.path.basename(src), []), *extra_flags, "-I", INCLUDE,
               "-I", CSRC, "-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return (os.path.basename(src), r.stderr)

    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 1)
        with concurrent.futures.ThreadPoolExecutor(n) as ex:
            for name, log in ex.map(compile_one, todo):
                if verbose and log.strip():
                    print(f"[{name}]\n{log}", file=sys.stderr)
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", "-rpath", "-Xlinker", os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
