"""In-tree build of libcello_gpu.so for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel into _build/, then
linked into the package directory.  The float64 kernels are compiled without
FMA contraction (-fmad=false) so their rounding follows the formulas term by
term; the float32 sweep keeps contraction.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libcello_gpu.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", INCLUDE, "-I", CSRC]
UNITS = {
    # float32 bulk path: hardware-approximate division and square root
    "k_f32.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "k_f64.cu": ["-fmad=false"],
    "k_de_f32.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "k_de_f64.cu": ["-fmad=false"],
    "table.cu": [],
    "mesh.cu": [],
    "noalloc.cu": [],
    "opcount.cu": [],
    "peak.cu": [],
    "particles.cu": ["-fmad=false"],
    "poisson.cu": ["-fmad=false"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def _compile(src: str, extra: list[str], verbose: bool) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every unit (only those out of date unless force) and link."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "cello.h"))
    jobs = []
    for src, extra in UNITS.items():
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or verbose or _stale(obj, [os.path.join(CSRC, src), *headers]):
            jobs.append((src, extra))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(lambda j: _compile(j[0], j[1], verbose), jobs))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in UNITS]
    if force or jobs or not os.path.exists(LIB):
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    return LIB


HOSTCHECK = os.path.join(BUILD, "libcello_hostcheck.so")


def build_hostcheck() -> str:
    """Host-compiled copy of the per-interface arithmetic and its adjoint
    (csrc/hostcheck.cu), used only by the CPU unit tests."""
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(CSRC, "hostcheck.cu")
    deps = [src] + [os.path.join(CSRC, f) for f in ("ppm.cuh", "adjoint.cuh", "opcount.cu", "cello_internal.h")]
    if _stale(HOSTCHECK, deps):
        cmd = [nvcc(), *ARCH, "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", CSRC,
               "-I", INCLUDE, "-shared", src, "-o", HOSTCHECK]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on hostcheck.cu:\n{r.stderr}")
    return HOSTCHECK


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
