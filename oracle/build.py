"""Build the plain-C FP64 oracle into a shared library (test infrastructure).

The oracle is compiled with -ffp-contract=off so that every product and sum
is rounded as written in the source.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tts_oracle.c")
LIB = os.path.join(HERE, "libtts_oracle.so")


def build(force: bool = False) -> str:
    hdr = os.path.join(HERE, "tts_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


def build_variant(defines, outdir) -> str:
    """Build a deliberately altered copy of the oracle (each entry of
    `defines` one ORC_PLANT_* switch) into outdir, for the tests that check
    a pin fails on a planted mistake.  Never used outside the test suite."""
    os.makedirs(outdir, exist_ok=True)
    out = os.path.join(outdir, "libtts_oracle_%s.so" % "_".join(d.lower() for d in defines))
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", *("-D" + d for d in defines), "-o", out, SRC, "-lm"]
    subprocess.check_call(cmd)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
