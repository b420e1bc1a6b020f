"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liblagp_oracle.so.

gcc -O2 -ffp-contract=off keeps every double operation separate (no fused
multiply-add), so results are the same on x86-64 and AArch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lagp_oracle.c")
LIB = os.path.join(HERE, "liblagp_oracle.so")


FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def compile_source(text: str, out_dir: str, name: str = "liblagp_oracle_variant.so") -> str:
    """Compile C source text (an altered copy of the oracle, for the tests that
    plant mistakes) with the oracle's flags into out_dir; returns the path."""
    src = os.path.join(out_dir, name.replace(".so", ".c"))
    with open(src, "w") as fh:
        fh.write(text)
    out = os.path.join(out_dir, name)
    subprocess.check_call(["gcc"] + FLAGS + ["-o", out, src, "-lm"])
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc"] + FLAGS + ["-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
