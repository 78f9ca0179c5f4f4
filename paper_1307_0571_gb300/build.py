"""Build libpms.so (the CUDA kernels and the C ABI) in-tree with nvcc for sm_103a.

Every translation unit compiles in parallel with one -gencode (compute_103a/sm_103a);
the result is paper_1307_0571_gb300/_build/libpms.so with the CUDA runtime linked
statically.  Nothing here runs on the GPU, so it works on a machine without one.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libpms.so")
SOURCES = ["pms_prep.cu", "pms_search_dna32.cu", "pms_search_dna64.cu", "pms_search_p5_32.cu",
           "pms_sort.cu", "pms_api.cu", "pms_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpms")


def _extra_flags() -> list[str]:
    """Extra nvcc flags from PMS_NVCC_FLAGS (e.g. -DPMS_SEARCH_MIN_BLOCKS=6), for tuning."""
    return os.environ.get("PMS_NVCC_FLAGS", "").split()


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    stamp = LIB + ".flags"
    if not os.path.exists(stamp) or open(stamp).read() != " ".join(_extra_flags()):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "pms.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "-I", os.path.join(ROOT, "include"), "-I", CSRC] + _extra_flags()

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(LIB + ".flags", "w") as f:
        f.write(" ".join(_extra_flags()))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
