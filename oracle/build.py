"""Compile the C part of the oracle into oracle/liboracle.so with gcc.

Building the checker is not using it: the package build step calls this so
that the tests find the library, but nothing on the engine's path loads it.
"""

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    out = os.path.join(_HERE, "liboracle.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        # one temporary file per process: processes that build at once each
        # replace the library atomically with a complete copy
        tmp = f"{out}.{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
