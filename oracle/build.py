"""Compile the CPU reference (``oracle.c``) into ``oracle/_build/liboracle.so``.

Test infrastructure: the tests, the smoke check and the benchmark's CPU
baseline load the result; the GPU library never does.  Plain C11 with
``-ffp-contract=off`` and no fast-math, so every ``fmaf`` and every separate
product in the source rounds exactly once, on x86-64 and on aarch64 alike.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c")]
HEADERS = [os.path.join(HERE, "oracle.h")]


def _stale():
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(p) > t for p in SOURCES + HEADERS + [__file__])


def build(force=False, verbose=False):
    """Build ``liboracle.so`` if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = [os.environ.get("CC", "gcc"), "-std=c11", "-O2", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp] + SOURCES + ["-lpthread", "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
