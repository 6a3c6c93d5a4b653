"""Build the FP64 oracle shared library (test infrastructure only).

The oracle is plain C compiled with gcc; it is the FP64 reference the CUDA
path is compared against, never a fallback for it.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline leg may load it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "iewpf_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile iewpf_oracle.c into liboracle.so next to it; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    # -ffp-contract=off keeps the arithmetic identical on x86_64 and aarch64
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
