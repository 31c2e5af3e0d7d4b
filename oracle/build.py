"""Build the FP64 CPU oracle (test infrastructure only).

Two shared objects are produced from the same source: a sequential build
(``liboracle.so``) and an OpenMP build over independent rows / columns
(``liboracle_omp.so``) used as the timed multi-core CPU baseline.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kzk_oracle.c")
FLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC", "-std=gnu11"]


def build(force: bool = False) -> None:
    for name, extra in (("liboracle.so", []), ("liboracle_omp.so", ["-fopenmp"])):
        out = os.path.join(HERE, name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        subprocess.check_call(["gcc", *FLAGS, *extra, SRC, "-o", out, "-lm"])


if __name__ == "__main__":
    build(force=True)
