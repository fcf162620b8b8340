"""In-tree build of libbbmd.so for sm_103a (nvcc, one -gencode, translation units in
parallel).  Output: paper_1105_5613_gb300/_build/libbbmd.so."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbbmd.so")
# (source, object, extra flags): k_force.cu is compiled once per block shape
SOURCES = [("bbmd_api.cu", "bbmd_api.o", []), ("k_sort.cu", "k_sort.o", []),
           ("k_integrate.cu", "k_integrate.o", []), ("k_observe.cu", "k_observe.o", []),
           ("k_probe.cu", "k_probe.o", [])] + \
          [("k_force.cu", f"k_force_z{z}.o", [f"-DBBMD_BLOCK_Z={z}"]) for z in (1, 2, 4, 8)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(HERE, "..", "include", "bbmd.h")] + \
        [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    return os.path.getmtime(obj) < max(os.path.getmtime(d) for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          out: str | None = None) -> str:
    """Compile the library; `out` (default _build/) and `extra` nvcc flags allow side builds
    of tuning variants."""
    OUT = out or globals()["OUT"]
    LIB = os.path.join(OUT, "libbbmd.so")
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    extra = extra or []

    def compile_one(entry) -> str:
        name, oname, defs = entry
        src = os.path.join(CSRC, name)
        obj = os.path.join(OUT, oname)
        if force or _stale(obj, src):
            cmd = [nvcc, *ARCH, *FLAGS, *defs, *extra, "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(map(os.path.getmtime, objs)):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
