"""Compile the FP64 CPU oracle (``mpm_oracle.c``) into ``liborcmpm.so``.

Test infrastructure: the oracle is what the CUDA path is checked against. It is
plain C, built with the host compiler, single threaded, and shares no source
with the CUDA library.

``build(openmp=True)`` compiles the same source with ``-fopenmp`` into
``liborcmpm_omp.so``: the all-core CPU baseline that bench.py times beside
the single-threaded oracle. The checker is always the serial library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mpm_oracle.c")
LIB = os.path.join(HERE, "liborcmpm.so")
LIB_OMP = os.path.join(HERE, "liborcmpm_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Build the oracle library (or its OpenMP build) if it is missing or older
    than its source; returns its path."""
    lib = LIB_OMP if openmp else LIB
    hdr = os.path.join(HERE, "mpm_oracle.h")
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    flags = ["-O3", "-fopenmp"] if openmp else ["-O2"]
    cmd = ["gcc"] + flags + ["-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> None:
    """The serial oracle, then its OpenMP build where the compiler has OpenMP
    (a warning otherwise: only the all-core baseline is then missing)."""
    build(force)
    try:
        build(force, openmp=True)
    except (subprocess.CalledProcessError, OSError) as e:
        sys.stderr.write("oracle: OpenMP build skipped (%s)\n" % e)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
    print(LIB)
