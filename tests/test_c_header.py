"""The public header is plain C: a C99 program includes it, links the library
and calls the host-only entry points (no GPU needed: version, status names,
argument errors, the uneven-batch plan)."""
import os
import shutil
import subprocess

import pytest

import paper_2410_22575_gb300 as cf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "chessfad.h"

int main(void)
{
    chessfad_config cfg;
    chessfad_request reqs[3] = {{CHESSFAD_ROSENBROCK, 4, 0, 0}, {CHESSFAD_ACKLEY, 8, 4, 0},
                                {CHESSFAD_FLETCHER_POWELL, 16, 12, 0}};
    chessfad_ragged_plan plan = 0;
    size_t ws = 0;
    long long ntiles = 0;
    int dummy = 0;
    if (chessfad_version() < 100) return 1;
    if (chessfad_hvp(7, 8, 4, 4, &dummy, &dummy, &dummy, NULL, CHESSFAD_FP64, NULL) != CHESSFAD_ERR_FUNCTION) return 2;
    if (chessfad_hvp(CHESSFAD_ACKLEY, 8, 4, 3, &dummy, &dummy, &dummy, NULL, CHESSFAD_FP64, NULL) != CHESSFAD_ERR_CHUNK)
        return 3;
    if (chessfad_default_config(CHESSFAD_ACKLEY, 64, 65536, CHESSFAD_FP32_COMP, &cfg) != CHESSFAD_SUCCESS) return 4;
    if (chessfad_ragged_plan_create(reqs, 3, CHESSFAD_FP32_COMP, 0, &plan) != CHESSFAD_SUCCESS) return 5;
    if (chessfad_ragged_plan_info(plan, &ws, &ntiles, NULL) != CHESSFAD_SUCCESS || ntiles != 3) return 6;
    chessfad_ragged_plan_destroy(plan);
    printf("%d %s|%d %d\n", chessfad_version(), chessfad_strerror(CHESSFAD_ERR_SIZE), cfg.csize, cfg.method);
    return 0;
}
"""


def test_c99_program_uses_the_header_and_library(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = cf.load()._name
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
           str(exe), lib, "-Wl,-rpath," + libdir]
    p = subprocess.run(cmd, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    version, rest = r.stdout.strip().split(" ", 1)
    assert int(version) == cf.chessfad_version()
    name, cfgs = rest.split("|")
    assert name == cf.strerror(-2)
    csize, method = (int(t) for t in cfgs.split())
    assert csize in (1, 2, 4, 8, 16, 32) and method in (0, 1)
