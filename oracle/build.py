"""Compile the FP64 CPU oracle (plain C, gcc + OpenMP) into oracle/liblbm_oracle.so.

Test infrastructure: the oracle is the correctness reference for the CUDA
library and is built here only so the tests and the CPU baseline can load it.
The source is compiled twice -- real (symbols orc_*) and complex (orcz_*) --
and both objects are linked into one shared library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cc = os.environ.get("CC", "gcc")
    flags = ["-O2", "-std=gnu11", "-fPIC", "-fopenmp", "-Wall", "-Wno-unused-function"]
    objs = []
    for tag, defs in (("r", []), ("z", ["-DORC_COMPLEX"])):
        obj = os.path.join(HERE, f"lbm_oracle_{tag}.o")
        cmd = [cc, *flags, *defs, "-c", SRC, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        objs.append(obj)
    tmp = LIB + ".tmp"
    subprocess.run([cc, "-shared", "-fopenmp", "-o", tmp, *objs, "-lm"], check=True)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
