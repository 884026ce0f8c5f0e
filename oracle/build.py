"""Compile the C oracle into ``oracle/_build/libgraph500_oracle.so`` and the
paper's multicore method (OpenMP) into ``oracle/_build/libgraph500_parallel.so``
with gcc.

Test infrastructure: the libraries it builds are loaded only by the tests, by
``__graft_entry__.smoke()`` and by the CPU legs of ``bench.py``.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "graph500_oracle.c")
SRC_PAR = os.path.join(HERE, "graph500_parallel.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgraph500_oracle.so")
LIB_PAR = os.path.join(OUT_DIR, "libgraph500_parallel.so")


def _compile(src, lib, flags, force):
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(src), os.path.getmtime(__file__))):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = lib + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc"] + flags + ["-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                                      "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Build the serial oracle library if it is missing or older than its source."""
    return _compile(SRC, LIB, ["-O2"], force)


def build_parallel(force: bool = False) -> str:
    """Build the OpenMP library of the paper's parallel method."""
    return _compile(SRC_PAR, LIB_PAR, ["-O3", "-fopenmp"], force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_parallel(force=True))
