"""Compile the FP64 CPU oracle (``mpm_oracle.c``) into ``liborcmpm.so``.

Test infrastructure: the oracle is what the CUDA path is checked against. It is
plain C, built with the host compiler, single threaded, and shares no source
with the CUDA library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mpm_oracle.c")
LIB = os.path.join(HERE, "liborcmpm.so")


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    hdr = os.path.join(HERE, "mpm_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
