"""Compile the CPU oracle (plain C) into oracle/liboracle.so.

Test infrastructure: the oracle is the checker of the CUDA tracker, built with
IEEE-strict flags (no contraction of a*b+c, no fast-math) so that its binary32
decision path is exactly the operation sequence written in tpc_oracle.c
(tpc_oracle_calib.c: the calibration chi2 and its gradient, binary64;
tpc_oracle_attach.c: the track-based cluster attachment;
tpc_oracle_compress.c: the cluster compression; tpc_oracle_loopers.c: the
looper-leg identification).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "tpc_oracle.c"), os.path.join(HERE, "tpc_oracle_calib.c"),
        os.path.join(HERE, "tpc_oracle_attach.c"), os.path.join(HERE, "tpc_oracle_compress.c"),
        os.path.join(HERE, "tpc_oracle_loopers.c")]
LIB = os.path.join(HERE, "liboracle.so")
FLAGS = ["-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
         "-fno-fast-math", "-fexcess-precision=standard", "-Wall"]


def build(force: bool = False) -> str:
    deps = [*SRCS, os.path.join(HERE, "tpc_oracle.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    tmp = f"{LIB}.{os.getpid()}.tmp"
    subprocess.run(["gcc", *FLAGS, *SRCS, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
