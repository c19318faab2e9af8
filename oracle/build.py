"""Compile the oracle's plain C sources into ``oracle/_build/liboracle_ct.so``.

ORACLE -- test infrastructure only.  Building the checker is not using it:
``__graft_entry__.build()`` calls :func:`build` so the tests find the library
on a fresh machine.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["sf_fan_oracle.c", "sf_helical_oracle.c"]
LIB = os.path.join(BUILD_DIR, "liboracle_ct.so")


def _has_openmp(cc: str) -> bool:
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        with open(src, "w") as f:
            f.write("#include <omp.h>\nint main(void){return omp_get_max_threads()>0?0:1;}\n")
        r = subprocess.run([cc, "-fopenmp", src, "-o", os.path.join(d, "t")], capture_output=True)
        return r.returncode == 0


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    if not force and os.path.exists(LIB):
        lib_mtime = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= lib_mtime for s in srcs):
            return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = os.environ.get("CC") or shutil.which("gcc") or "cc"
    flags = ["-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math", "-ffp-contract=off"]
    if _has_openmp(cc):
        flags.append("-fopenmp")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *flags, *srcs, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
