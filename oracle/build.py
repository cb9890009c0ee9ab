"""Build the FP64 CPU oracle shared library (test infrastructure only).

Compiles ``dg_oracle.c`` with gcc into ``oracle/_build/liboracle.so``.  OpenMP
is used when the compiler supports it; otherwise the oracle runs serially.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = os.path.join(HERE, "dg_oracle.c")


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
        err = r.stderr
    raise RuntimeError("oracle build failed:\n" + err)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
