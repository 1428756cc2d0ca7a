"""Build the in-tree CUDA library libnlinv.so for sm_103a with nvcc.

The host C ABI (csrc/nlinv.cu) is one translation unit; the kernels are
compiled once per FFT grid size from csrc/grid.cu (the sizes listed by
NLINV_GRIDS in csrc/common.h), all units in parallel, then linked into one
shared library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libnlinv.so")
OBJ = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def grid_sizes():
    """(G1, G2, N, TW, MINB) of every compiled grid, as NLINV_GRIDS in csrc/common.h lists them."""
    txt = open(os.path.join(CSRC, "common.h")).read()
    body = re.search(r"#define NLINV_GRIDS\(X\)((?:.*\\\n)*.*)", txt).group(1)
    return [tuple(int(v) for v in m)
            for m in re.findall(r"X\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", body)]


def deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "nlinv.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps())


def units(extra=(), sizes=None, obj=OBJ):
    """(object path, nvcc compile command) of every translation unit."""
    base = [nvcc(), *FLAGS, *ARCH, *extra, "-I", INCLUDE, "-I", CSRC, "-c"]
    out = [(os.path.join(obj, "nlinv.o"), base + [os.path.join(CSRC, "nlinv.cu")])]
    for g1, g2, n, tw, mb in (sizes or grid_sizes()):
        o = os.path.join(obj, f"grid_{g1}x{g2}_{n}.o")
        out.append((o, base + [f"-DNLINV_G1={g1}", f"-DNLINV_G2={g2}", f"-DNLINV_NR={n}", f"-DNLINV_TWU={tw}",
                               f"-DNLINV_MINBU={mb}", os.path.join(CSRC, "grid.cu")]))
    return out


def build(force: bool = False, verbose: bool = False, extra=(), sizes=None, lib: str = LIB, obj: str = OBJ,
          workers: int = 0) -> str:
    """Compile every unit (in parallel) and link libnlinv.so (static cudart).
    `sizes` restricts the grid sizes (quick builds; the others are then
    unsupported), `extra` adds nvcc flags, `lib` names the output, `obj` the
    folder of the objects (one per concurrent build), `workers` caps the
    parallel compilers (0: one per core)."""
    if not force and lib == LIB and not extra and sizes is None and up_to_date():
        return lib
    os.makedirs(obj, exist_ok=True)
    jobs = units(extra, sizes, obj)

    def run(job):
        o, cmd = job
        cmd = cmd + ["-o", o]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        return o

    cap = workers if workers > 0 else (os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), cap))) as ex:
        objs = list(ex.map(run, jobs))
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *objs], check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    build(force=True, verbose=True)
