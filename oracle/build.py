"""Compile the oracle's C library (test infrastructure; see oracle/__init__.py).

``python -m oracle.build`` or ``oracle.build.build()`` writes
``oracle/_build/libkfvm_oracle.so``.  Plain gcc, no CUDA.  ``-ffp-contract=off``
keeps every multiply and add a separately rounded IEEE operation, so the oracle
gives the same bits on x86_64 and aarch64.

``build(threaded=True)`` writes a second library, ``libkfvm_oracle_omp.so``,
from the same source with ``-fopenmp``: the cell loops are shared out over the
host's cores, each cell computed by the same statements, so its results equal
the single-threaded library's.  It exists only to time the oracle on every
host core; the pins and parity tests use the single-threaded library.
"""
from __future__ import annotations

import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kfvm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkfvm_oracle.so")
LIB_OMP = os.path.join(OUT_DIR, "libkfvm_oracle_omp.so")


def build(force: bool = False, threaded: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    out = LIB_OMP if threaded else LIB
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11"]
    if threaded:
        cmd.append("-fopenmp")
    cmd += ["-o", out + ".tmp", SRC, "-lm"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        cmd.append("-lquadmath")
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(force=True))
    print(build(force=True, threaded=True))
