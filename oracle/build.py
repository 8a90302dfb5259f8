"""Build the CPU oracle's two shared libraries (float and double) with gcc.

Test infrastructure: the product library never links these.  Flags keep
IEEE semantics (no fast-math, no FMA contraction) so the float build takes
every threshold decision in single precision exactly as written.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gs_oracle.c")
OUT = os.path.join(HERE, "_build")
LIBS = {"f32": "liborc_f32.so", "f64": "liborc_f64.so"}


def lib_path(kind: str) -> str:
    return os.path.join(OUT, LIBS[kind])


def build(force: bool = False) -> None:
    os.makedirs(OUT, exist_ok=True)
    for kind, name in LIBS.items():
        dst = os.path.join(OUT, name)
        if not force and os.path.exists(dst) and os.path.getmtime(dst) >= os.path.getmtime(SRC):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", SRC, "-o", dst + ".tmp", "-lm"]
        if kind == "f64":
            cmd.insert(1, "-DORC_DOUBLE")
        subprocess.run(cmd, check=True)
        os.replace(dst + ".tmp", dst)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print("oracle built:", [lib_path(k) for k in LIBS])
