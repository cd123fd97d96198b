"""Compile the C oracle (test infrastructure) into oracle/_build/liboracle.so."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = [os.path.join(HERE, "apo_oracle.c")]
DEPS = SRC + [os.path.join(HERE, f) for f in ("vote_program.inc", "midpoint.inc", "exactphi.inc", "fourd.inc")]
# No FMA contraction, no fast-math, rounding-mode-aware code generation.
CFLAGS = ["-O1", "-std=c11", "-frounding-math", "-ffp-contract=off", "-fno-fast-math",
          "-fno-builtin", "-fopenmp", "-shared", "-fPIC", "-Wall", "-Wno-unknown-pragmas"]


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t_lib = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t_lib for p in DEPS):
            return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *CFLAGS, *SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
