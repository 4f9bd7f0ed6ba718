"""Build the CUDA library libcx.so in-tree for sm_103a.

Each .cu file under csrc/ is compiled to an object in parallel, then nvcc
links the objects into paper_1301_5058_gb300/libcx.so (CUDA runtime linked
statically, so the library needs only the driver at run time).  The
instantiation units (*_inst.cu) are compiled once per (precision,
chemotaxis law, mobility), so that the largest sets of kernels compile in
parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcx.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC] + ARCH


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcx.so")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


# (precision, chemotaxis law, mobility) combinations of an instantiation unit
INST_DEFINES = [(p, law, mob) for p in (0, 1) for law in (0, 1) for mob in (0, 1)]


def _jobs():
    """(source, object, extra flags) for every compilation."""
    jobs = []
    for src in _sources():
        base = os.path.basename(src)[:-3]
        if base.endswith("_inst"):
            for p, law, mob in INST_DEFINES:
                jobs.append((src, os.path.join(BUILD, f"{base}_p{p}l{law}m{mob}.o"),
                             [f"-DCX_INST_PREC={p}", f"-DCX_INST_LAW={law}", f"-DCX_INST_MOB={mob}"]))
        else:
            jobs.append((src, os.path.join(BUILD, base + ".o"), []))
    return jobs


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile csrc/*.cu and link libcx.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs = _jobs()

    def compile_one(job):
        src, obj, defs = job
        cmd = [cc, "-c", src, "-o", obj] + NVCC_FLAGS + defs + list(extra_flags)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(obj)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    # the biggest units first, so that they start before the small ones
    jobs.sort(key=lambda j: -os.path.getsize(j[0]) - (1 << 20) * bool(j[2]))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 8, len(jobs)))) as ex:
        objs = list(ex.map(compile_one, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "-v" in sys.argv else []))
