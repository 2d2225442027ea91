"""Build the CUDA library ``_build/libchessfad.so`` for sm_103a, in-tree.

Each translation unit under ``csrc/`` is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` (``instances.cu``
once per (function, precision) slice) and the objects are linked into one
shared library with the CUDA runtime linked statically.
A rebuild happens only when a source or the public header is newer than the
library.  Usage: ``python -m paper_2410_22575_gb300.build [--force]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libchessfad.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-fvisibility=hidden"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libchessfad")


# instances.cu is compiled once per (function, precision) slice.
SLICED = "instances.cu"
SLICES = [(fn, f64) for fn in (0, 1, 2) for f64 in (0, 1)]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def compile_units() -> list[tuple[str, list[str], str]]:
    """(source, extra flags, object name) of every translation unit."""
    units = []
    for src in sources():
        base = os.path.basename(src)[:-3]
        if os.path.basename(src) == SLICED:
            for fn, f64 in SLICES:
                units.append((src, [f"-DCHESSFAD_SLICE_FN={fn}", f"-DCHESSFAD_SLICE_F64={f64}"],
                              f"{base}_{fn}_{f64}.o"))
        else:
            units.append((src, [], base + ".o"))
    return units


def _deps() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


# Sources compiled at run time (NVRTC) for user-supplied functions, embedded
# in the library as string constants: (C++ name, file under csrc/).
EMBEDDED = (("kHdualSrc", "hdual.cuh"), ("kSymLayoutSrc", "sym_layout.cuh"), ("kUserNumSrc", "user_num.cuh"),
            ("kUserKernelSrc", "user_kernel.cuh"))
DELIM = "CHESSFAD_EMBED"


def write_embedded() -> str:
    """Write _build/user_embed.h: each run-time-compiled source as a raw string."""
    lines = ["// Generated by build.py from csrc/: sources compiled at run time by NVRTC.", "#pragma once"]
    for cname, fname in EMBEDDED:
        text = open(os.path.join(CSRC, fname)).read()
        if f"){DELIM}" in text:
            raise RuntimeError(f"{fname} contains the raw-string delimiter")
        lines.append(f'static const char {cname}[] = R"{DELIM}({text}){DELIM}";')
    path = os.path.join(OUT, "user_embed.h")
    body = "\n".join(lines) + "\n"
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)
    return path


def _compile(unit: tuple[str, list[str], str], verbose_ptxas: bool) -> tuple[str, str]:
    src, extra, name = unit
    obj = os.path.join(OUT, name)
    cmd = ([nvcc()] + ARCH + FLAGS + extra + ["-I", OUT] + (["-Xptxas", "-v"] if verbose_ptxas else [])
           + ["-c", src, "-o", obj])
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{p.stdout}\n{p.stderr}")
    return obj, p.stderr


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    write_embedded()
    units = compile_units()
    # the slowest units first, so the parallel build ends sooner
    order = {"ragged": 0, "instances": 1}
    units.sort(key=lambda u: order.get(os.path.basename(u[0])[:-3], 2))
    jobs = jobs or min(len(units), max(1, os.cpu_count() or 1))
    logs = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for obj, log in ex.map(lambda u: _compile(u, verbose_ptxas), units):
            logs.append((obj, log))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in logs] + ["-cudart", "static", "-ldl"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    if verbose_ptxas:
        with open(os.path.join(OUT, "ptxas.log"), "w") as f:
            for obj, log in logs:
                f.write(f"== {os.path.basename(obj)}\n{log}\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
