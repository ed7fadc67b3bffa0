"""Compile the FP64 oracle (plain C) into oracle/_build/liboracle.so.

Test infrastructure only: the oracle is the reference the CUDA path is
checked against; building it does not make the product depend on it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "lbm_oracle.c"), os.path.join(HERE, "lbm3d_oracle.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if the shared library is missing or stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = SRCS + [os.path.join(HERE, "lbm_oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    # -ffp-contract=off: no fused multiply-adds, so the FP64 arithmetic is the
    # plain sequence of operations written in the source on every host.
    # -fopenmp runs the independent per-cell passes on every core (results
    # are bit-identical on any thread count); without OpenMP it runs on one.
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
           "-fPIC", "-shared"] + SRCS + ["-o", tmp, "-lm"]
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], stdout=subprocess.DEVNULL,
                      stderr=subprocess.DEVNULL).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
