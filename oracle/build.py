"""Compile the CPU oracle (plain C) into a shared library under oracle/_build/.

Test infrastructure only: the product library never loads what this builds.  The build
uses the system C compiler with OpenMP when it is available (the per-island loops of the
oracle are independent within a generation), otherwise a serial build.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ga_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "libga_oracle.so")


def _compile(extra):
    # -ffp-contract=off: every float operation is rounded on its own (no fused multiply-add),
    # as the normal-deviate arithmetic requires
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra, SRC,
           "-o", OUT, "-lm"]
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= os.path.getmtime(SRC)
            and os.path.getmtime(OUT) >= os.path.getmtime(__file__)):
        return OUT
    res = _compile(["-fopenmp"])
    if res.returncode != 0:
        res = _compile([])
    if res.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + res.stderr)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
