"""Compile the CPU oracle (plain C) into ``oracle/liboracle.so`` with gcc.

Test infrastructure: building the checker is not using it.  No fused
multiply-add (-ffp-contract=off) so the oracle rounds the same way on x86-64
and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(HERE, "liboracle.so")


def build() -> str:
    out = library_path()
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
           "-o", tmp, os.path.join(HERE, "bilu_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build())
