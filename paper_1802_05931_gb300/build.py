"""Build libddqmc.so in place with nvcc for sm_103a (GB300).

One translation unit, one -gencode, static CUDA runtime (so the library loads
on a machine without a GPU), no FMA contraction in host or device code (the
fixed-point rate thresholds are bit-exact functions of IEEE double operations).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libddqmc.so")
SOURCES = ["ddqmc_api.cu"]
DEPS = ["ddqmc_api.cu", "common.cuh", "spawn.cuh", "radix.cuh", "merge.cuh", "finalize.cuh", "transfer.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_command(out):
    # host code: no contraction (its fixed-point rate tables must equal the
    # oracle's); device code does its floating point with explicitly rounded
    # intrinsics, or in single products whose integer result is corrected
    return ["nvcc", "-std=c++17", "-O3", ARCH, "-lineinfo",
            "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", "-cudart", "static", "-lpthread",
            "-o", out] + [os.path.join(CSRC, s) for s in SOURCES]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, d) for d in DEPS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "ddqmc.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False) -> str:
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run(nvcc_command(tmp), check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
