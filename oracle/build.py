"""Compile the CPU oracle (oracle.c) into ``oracle/liboracle.so`` with plain gcc.

The oracle is test infrastructure: this builds the checker, nothing more.
``-ffp-contract=off`` keeps every multiply and add separately rounded (gcc
would otherwise fuse them into FMAs on aarch64), so the oracle computes the
plain IEEE expressions it is written as.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, "oracle.c")]


def build(force: bool = False) -> str:
    deps = SRC + [os.path.join(HERE, "oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in deps)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp] + SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
