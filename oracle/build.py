"""Build the FP64 C oracle into oracle/_build/liblbm_oracle.so.

Test infrastructure only: the oracle is loaded by the tests, the smoke check and the
CPU-baseline leg of bench.py, never by the CUDA library or its Python binding.
The oracle is compiled with -ffp-contract=off (no fused multiply-add), and with
OpenMP over lattice rows when the compiler supports it (the rows of one stage are
independent, so the result does not depend on the thread count).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, SRC, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
