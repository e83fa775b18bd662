"""Build step of the CPU oracle: ``gcc -O2 -shared`` of mbr_oracle.c into liboracle.so (in-tree).

Plain IEEE double arithmetic: no -ffast-math, no -march flags, so the x86 and Arm builds agree.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mbr_oracle.c")
SRC_SDF = os.path.join(HERE, "sdf_oracle.c")
HDR = os.path.join(HERE, "mbr_oracle.h")


def library_path():
    return os.path.join(HERE, "liboracle.so")


def build(force=False):
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(SRC), os.path.getmtime(SRC_SDF), os.path.getmtime(HDR)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter",
           "-o", tmp, SRC, SRC_SDF, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
