"""Compile the FP64 C oracle into ``oracle/libiqa_oracle.so`` (test infrastructure).

Plain gcc, ``-O2 -ffp-contract=off`` and no fast-math, so every floating-point
operation in ``iqa_oracle.c`` happens as written.  OpenMP is used when the
compiler has it; it only spreads whole tiles over threads.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "iqa_oracle.c")
LIB = os.path.join(HERE, "libiqa_oracle.so")


def build(force=False, verbose=False):
    """Build the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
            "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), r.stdout, r.stderr)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def build_from_source(src_text, out_path, openmp=False):
    """Compile an alternative oracle source text (used by the mutation tests,
    which plant mistakes in a copy of the oracle) into ``out_path``."""
    src_path = out_path + ".c"
    with open(src_path, "w") as f:
        f.write(src_text)
    cmd = ["gcc"] + (["-fopenmp"] if openmp else []) + [
        "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC",
        "-shared", src_path, "-o", out_path, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("mutant build failed:\n" + r.stderr)
    return out_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
