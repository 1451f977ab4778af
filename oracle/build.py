"""Compile the C++17 oracle into ``oracle/_build/liboracle.so`` (test infrastructure only).

-ffp-contract=off keeps the geometric arithmetic (d, r, k*r, d.n) in the written order so the
arguments of the Hankel functions are reproducible.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def library_path(tag=""):
    return os.path.join(HERE, "_build", f"liboracle{tag}.so")


def build(extra_flags=(), tag="", out=None):
    src = os.path.join(HERE, "wsbm_oracle.cpp")
    out = out or library_path(tag)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", *extra_flags, "-o", out, src]
    subprocess.run(cmd, check=True)
    return out


if __name__ == "__main__":
    print(build())
