"""Compiles the FP64 oracle (plain C) into oracle/liboracle.so with gcc.

Building the checker is not using it: ``__graft_entry__.build()`` calls this so
that the oracle exists on any machine the tests run on.
"""

from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "ldpc_oracle.c")
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src,
                           "-lm", "-lpthread"])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
