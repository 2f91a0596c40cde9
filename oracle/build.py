"""Compile the C oracle (``sr_oracle.c``) into ``liboracle.so`` beside it.

Test infrastructure only: the oracle is the slow, obviously correct CPU
statement of the device-wide sum.  Plain ``gcc -O2`` with no target-specific
flags, so the same source gives the same results on x86_64 and aarch64 hosts.
Strict IEEE semantics (no -ffast-math, no FMA contraction) keep the FP64
loops a literal sequential sum.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sr_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
