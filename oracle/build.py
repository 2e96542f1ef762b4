"""Compile the oracle's C code into oracle/_build/libhk_oracle.so.

Test infrastructure: the oracle is built so the test-suite can check the CUDA
path against it; nothing on the product path loads it.  The flags keep binary64
arithmetic exactly as written: -ffp-contract=off forbids fused multiply-add
(GCC fuses by default in GNU mode, notably on aarch64), and no fast-math
option is given.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hk_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhk_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared", "-pthread"]


def build(force: bool = False) -> str:
    """Build the library if missing or older than its source; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
