"""Compile tpcgen/helix.c (exact helix/plane crossings) into tpcgen/libhelix.so."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "helix.c")
LIB = os.path.join(HERE, "libhelix.so")


def build(force: bool = False) -> str:
    deps = [SRC, os.path.abspath(__file__)]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    tmp = f"{LIB}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp", SRC, "-o", tmp,
                    "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
