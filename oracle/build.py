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


def build(force: bool = False, variant: str = "", defines=()) -> str:
    """Builds liboracle.so, or liboracle_<variant>.so compiled with extra -D defines (the
    tests' reference variants)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = LIB if not variant else os.path.join(OUT_DIR, "liboracle_%s.so" % variant)
    if not force and os.path.exists(lib):
        t_lib = os.path.getmtime(lib)
        if all(os.path.getmtime(p) <= t_lib for p in DEPS):
            return lib
    cc = os.environ.get("CC", "gcc")
    tmp = lib + ".tmp%d" % os.getpid()
    extra = ["-D" + d for d in defines] + (["-Wno-unused-function"] if defines else [])
    cmd = [cc, *CFLAGS, *extra, *SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
