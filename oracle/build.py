"""Compile the oracle's C library (test infrastructure; see oracle/__init__.py).

``python -m oracle.build`` or ``oracle.build.build()`` writes
``oracle/_build/libkfvm_oracle.so``.  Plain gcc, no CUDA.  ``-ffp-contract=off``
keeps every multiply and add a separately rounded IEEE operation, so the oracle
gives the same bits on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kfvm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkfvm_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11", "-o", LIB + ".tmp", SRC, "-lm"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        cmd.append("-lquadmath")
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
