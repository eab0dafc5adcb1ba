"""Compile the CPU oracle (plain C, gcc) into ``oracle/liboracle.so``.

TEST INFRASTRUCTURE ONLY: the oracle is what the CUDA library is checked
against; only the tests, the smoke check and the CPU-baseline leg of the bench
load it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["philox.c", "ising.c", "sw.c", "wl.c", "on.c", "ea_pt.c"]
HEADERS = ["oracle.h", "lattice.h"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def build(force=False):
    """Build the oracle library if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-ffp-contract=off",
           "-fPIC", "-shared", "-o", tmp] + [os.path.join(HERE, f) for f in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
