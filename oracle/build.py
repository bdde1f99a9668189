"""Compile the CPU oracle (oracle.c) into liboracle.so next to this file.

Test infrastructure only.  Flags keep every float32 operation rounded on its
own: no fused multiply-add contraction, no fast-math.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "oracle.c")]
HDR = [os.path.join(HERE, "oracle.h")]
LIB = os.path.join(HERE, "liboracle.so")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
          "-fPIC", "-shared", "-Wall", "-Wextra"]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in SRC + HDR + [os.path.abspath(__file__)])


def build(force: bool = False) -> str:
    """Builds with OpenMP (the *_threads functions then use several host
    threads); without it if the compiler lacks OpenMP."""
    if force or stale():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, "-fopenmp", "-o", tmp, *SRC, "-lm"]
        if subprocess.run(cmd, capture_output=True).returncode != 0:
            subprocess.run(["gcc", *CFLAGS, "-o", tmp, *SRC, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
