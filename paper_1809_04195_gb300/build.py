"""Build libt2sh.so for sm_103a with nvcc (one object per translation unit, compiled in
parallel, then linked).  Output: ``paper_1809_04195_gb300/libt2sh.so``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libt2sh.so")
SOURCES = ["t2sh_api.cu", "k_prep.cu", "k_fft.cu", "k_fft_fast.cu", "k_col_tma.cu", "k_col_tc.cu", "k_col_pr.cu", "k_fused.cu", "k_llr.cu", "k_cg.cu", "k_post.cu", "k_wavelet.cu", "k_preproc.cu", "t2sh_preproc.cu", "t2sh_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _compile(src: str, extra: list[str]) -> str:
    out = os.path.join(OBJ, src.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return out + ("\n" + r.stderr if r.stderr.strip() else "")


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile every CUDA source and link libt2sh.so; returns the library path."""
    os.makedirs(OBJ, exist_ok=True)
    extra = list(extra or [])
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(os.path.dirname(PKG), "include", "t2sh.h"))
    newest = max(os.path.getmtime(f) for f in srcs + hdrs + [__file__])
    if not extra and os.path.exists(LIB) and os.path.getmtime(LIB) > newest:
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    objs = [r.split("\n", 1)[0] for r in res]
    if verbose:
        for r in res:
            if "\n" in r:
                print(r.split("\n", 1)[1], file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose=v, extra=["-Xptxas", "-v"] if v else None))
