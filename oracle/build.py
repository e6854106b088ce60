"""Compile the oracle's C code into oracle/_lib/liboracle.so (gcc, OpenMP).

The flags pin plain IEEE double semantics: no fused multiply-add contraction,
no fast-math reassociation.
"""

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def build(verbose: bool = False) -> str:
    out_dir = os.path.join(_HERE, "_lib")
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(_HERE, "oracle.c")
    out = os.path.join(out_dir, "liboracle.so")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", out, src, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
