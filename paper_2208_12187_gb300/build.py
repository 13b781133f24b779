"""In-tree build of libgbfit.so for sm_103a (nvcc, no CMake).

Each translation unit is compiled in parallel, then linked into
paper_2208_12187_gb300/_build/libgbfit.so.  Rebuilds only when a source or
header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libgbfit.so")
SOURCES = ["kernels_mixed.cu", "kernels_mixed_eval.cu", "kernels_fp64.cu", "kernels_fp64_eval.cu", "kernels_single.cu",
           "kernels.cu", "engine.cu", "user_models.cu",
           "cov_kernels.cu"]
# device headers embedded in the library for run-time compilation of user models
RTC_HEADERS = ["rtc_compat.cuh", "gbfit_internal.cuh", "sync_device.cuh", "models.cuh", "trf_device.cuh", "trf_step.cuh",
               "round_kernels.cuh", "user_model.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", INCLUDE, "-I", BUILD]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbfit")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "gbfit.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def write_rtc_headers() -> None:
    """_build/rtc_headers.inc: the device headers as C string literals (names and sources)."""
    delim = "GBFIT_RTC"
    parts = ["// generated by build.py from csrc/ (do not edit)", f"static const int k_rtc_count = {len(RTC_HEADERS)};",
             "static const char* const k_rtc_names[] = {" + ", ".join(f'"{h}"' for h in RTC_HEADERS) + "};",
             "static const char* const k_rtc_srcs[] = {"]
    for h in RTC_HEADERS:
        with open(os.path.join(CSRC, h)) as f:
            text = f.read()
        if f"){delim}" in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        parts.append(f'R"{delim}({text}){delim}",')
    parts.append("};")
    out = os.path.join(BUILD, "rtc_headers.inc")
    tmp = out + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(parts) + "\n")
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile libgbfit.so for sm_103a; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    write_rtc_headers()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
