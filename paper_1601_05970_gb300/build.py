"""Build libfftg.so in-tree with nvcc for sm_103a.

The pass kernels (small and finite strain) are compiled once per supported
grid size, in parallel, and linked with the host drivers into one shared
library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfftg.so")

GRIDS = (3, 5, 9, 15, 25, 27, 45, 75, 81, 125, 135, 225, 243)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile (if sources changed) and return the path of libfftg.so."""
    os.makedirs(BUILD, exist_ok=True)
    digest = _sources_digest()
    stamp = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return LIB
    nvcc = _nvcc()
    jobs = jobs or max(1, min(16, os.cpu_count() or 1))
    units = []
    for n in GRIDS:
        units.append(([nvcc] + ARCH + FLAGS + [f"-DFFTG_N={n}", "-c",
                       os.path.join(CSRC, "passes_inst.cu"), "-o",
                       os.path.join(BUILD, f"passes_{n}.o")]))
        units.append(([nvcc] + ARCH + FLAGS + [f"-DFFTG_N={n}", "-c",
                       os.path.join(CSRC, "passes_tune.cu"), "-o",
                       os.path.join(BUILD, f"tune_{n}.o")]))
        units.append(([nvcc] + ARCH + FLAGS + [f"-DFFTG_N={n}", "-c",
                       os.path.join(CSRC, "fs_inst.cu"), "-o",
                       os.path.join(BUILD, f"fs_{n}.o")]))
    units.append([nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, "finite_strain.cu"), "-o",
                                          os.path.join(BUILD, "finite_strain.o")])
    units.append([nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, "api.cu"), "-o",
                                          os.path.join(BUILD, "api.o")])
    units.append([nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, "noalloc.cu"), "-o",
                                          os.path.join(BUILD, "noalloc.o")])
    units.append([nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, "server.cu"), "-o",
                                          os.path.join(BUILD, "server.o")])
    units.append([nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, "probe.cu"), "-o",
                                          os.path.join(BUILD, "probe.o")])
    # the schedule cache is keyed by this build's source digest
    units.append([nvcc] + ARCH + FLAGS + [f'-DFFTG_BUILD_ID="{digest[:16]}"', "-c",
                                          os.path.join(CSRC, "autotune.cu"), "-o",
                                          os.path.join(BUILD, "autotune.o")])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for out in ex.map(_run, units):
            logs.append(out)
    objs = ([os.path.join(BUILD, f"passes_{n}.o") for n in GRIDS]
            + [os.path.join(BUILD, f"tune_{n}.o") for n in GRIDS]
            + [os.path.join(BUILD, f"fs_{n}.o") for n in GRIDS]
            + [os.path.join(BUILD, "finite_strain.o"), os.path.join(BUILD, "api.o"), os.path.join(BUILD, "noalloc.o"),
               os.path.join(BUILD, "server.o"), os.path.join(BUILD, "probe.o"),
               os.path.join(BUILD, "autotune.o")])
    tmp = LIB + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(digest)
    if verbose:
        sys.stdout.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
