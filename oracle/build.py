"""Compile the FP64 CPU oracle (test infrastructure; see bfibm_oracle.c).

Two builds of the same source: ``liboracle_st.so`` (one thread, the plain
reference) and ``liboracle_omp.so`` (OpenMP over the independent loops; every
reduction stays serial, so both give identical results).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bfibm_oracle.c")
OUT = os.path.join(HERE, "_build")

FLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
         "-D_GNU_SOURCE", "-Wall", "-Wno-unknown-pragmas"]


def lib_path(omp=False):
    return os.path.join(OUT, "liboracle_omp.so" if omp else "liboracle_st.so")


def build(force=False, omp_too=True):
    os.makedirs(OUT, exist_ok=True)
    targets = [(lib_path(False), [])]
    if omp_too:
        targets.append((lib_path(True), ["-fopenmp"]))
    for out, extra in targets:
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        tmp = out + ".tmp%d" % os.getpid()
        cmd = ["gcc"] + FLAGS + extra + ["-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return lib_path(False)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(lib_path(False))
