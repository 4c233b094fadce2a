"""Compile the oracle's plain C fingerprint (crac_fp.c) with gcc.

TEST INFRASTRUCTURE ONLY: builds the checker, not the product.  The output
goes to oracle/_lib/ (git-ignored) and is rebuilt on each machine, since the
CPU and GPU hosts differ in architecture.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "crac_fp.c")
OUT_DIR = os.path.join(HERE, "_lib")
OUT = os.path.join(OUT_DIR, "liboracle_fp.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = OUT + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, SRC], check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
