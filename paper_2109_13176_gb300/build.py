"""Builds libgvom.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2109_13176_gb300/_build/libgvom.so with the CUDA runtime linked
statically, so the library needs nothing but the NVIDIA driver at run time.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgvom.so")
LIB_CHECKED = os.path.join(BUILD, "checked", "libgvom_checked.so")
SOURCES = ["ingest.cu", "extract.cu", "export.cu", "api.cu", "batch.cu", "pipeline.cu", "microbench.cu", "noalloc.cu",
           "selftest.cu"]
HEADERS = ["gvom_internal.h", "device_sync.cuh", "exact_convert.cuh", os.path.join("..", "..", "include", "gvom.h"),
           os.path.join("..", "..", "include", "gvom_microbench.h"),
           os.path.join("..", "..", "include", "gvom_selftest.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          checked: bool = False) -> str:
    """Builds libgvom.so, or with checked=True the range-checked debug
    variant _build/checked/libgvom_checked.so (GVOM_CHECKED: every computed
    index is checked in the kernels and a violation reported as
    GVOM_ERR_BOUNDS); returns the library's path."""
    out_dir = os.path.join(BUILD, "checked") if checked else BUILD
    lib_path = LIB_CHECKED if checked else LIB
    if checked:
        extra_flags = [*(extra_flags or []), "-DGVOM_CHECKED=1"]
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS]
    objs, procs = [], []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [sp, *headers, __file__]):
            cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *(extra_flags or []), "-c", sp, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out.decode(errors='replace')}")
        if verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if force or procs or _stale(lib_path, objs):
        tmp = lib_path + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout.decode(errors='replace')}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
