"""Build step for the CPU oracle (test infrastructure only).

Compiles ``trsm_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc.
``-ffp-contract=off`` keeps every ``a*b + c`` rounded twice, the canonical
IEEE reading the oracle is written against.  OpenMP is used when the compiler
offers it (the columns of X are independent); without it the oracle runs on
one thread and says so through ``oracle_max_threads``.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "trsm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
            "-fno-fast-math", SRC, "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), r.returncode, r.stderr[-2000:])
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr[-4000:])


if __name__ == "__main__":
    print(build(force=True, verbose=True))
