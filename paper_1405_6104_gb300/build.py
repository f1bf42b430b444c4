"""Compiles the CUDA library (sm_103a) in-tree: one object per source file,
compiled in parallel, linked into ``_build/libvpath.so``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libvpath.so")
SOURCES = ["vp_rebuild.cu", "vp_pair.cu", "vp_cv.cu", "vp_update.cu", "vp_capi.cu", "vp_noalloc.cu", "vp_adjoint.cu",
           "vp_toy2d.cu", "vp_contacts.cu", "vp_step.cu"]
HEADERS = ["vp_internal.cuh", "vp_dev.cuh", "vp_cvpair.cuh", "vp_adjoint.cuh", "vp_contacts.cuh", "vp_pair_dev.cuh",
           "vp_cv_dev.cuh", "vp_rebuild_dev.cuh", "vp_update_dev.cuh", os.path.join("..", "..", "include", "vpath.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden"]
# the pair kernel works far from the denormal range: flush-to-zero keeps its
# reciprocal square root a single instruction
EXTRA = {"vp_pair.cu": ["-ftz=true"],
         # the toy model runs FP64 in the operation order of its equations
         "vp_toy2d.cu": ["-fmad=false"]}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(SRC, s) for s in SOURCES]
    hdrs = [os.path.normpath(os.path.join(SRC, h)) for h in HEADERS]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest(srcs + hdrs + [__file__]):
        return LIB
    nvcc = _nvcc()

    # objects of this process only (several processes may build at once; the
    # library itself is replaced atomically)
    objdir = os.path.join(OUT, f"obj.{os.getpid()}")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *EXTRA.get(os.path.basename(src), []), "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, log in results:
            print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results] + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    for o, _ in results:
        os.remove(o)
    os.rmdir(objdir)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
