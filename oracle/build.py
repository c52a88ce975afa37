"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so,
and its operation counter into oracle/op_count.

Plain gcc, no shared headers with the CUDA path.  ``-ffp-contract=off`` keeps
the rounding identical on x86_64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")
OPC_SRC = os.path.join(HERE, "op_count.cpp")
OPC_BIN = os.path.join(HERE, "op_count")


def _stale(out: str, *srcs: str) -> bool:
    return not os.path.exists(out) or any(os.path.getmtime(out) < os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    """liboracle.so, its OpenMP build liboracle_omp.so (same source, same
    bits, nodes shared among threads), and the operation counter op_count
    (lbm_oracle.c traced in C++, see op_count.cpp)."""
    for out, extra in ((LIB, ["-Wno-unknown-pragmas"]), (LIB_OMP, ["-fopenmp"])):
        if force or _stale(out, SRC):
            tmp = out + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                   "-shared", "-Wall", "-Wextra"] + extra + ["-o", tmp, SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
    if force or _stale(OPC_BIN, SRC, OPC_SRC):
        tmp = OPC_BIN + ".tmp%d" % os.getpid()
        subprocess.run(["g++", "-O1", "-std=c++17", "-Wall", "-Wno-unknown-pragmas", "-o", tmp, OPC_SRC], check=True)
        os.replace(tmp, OPC_BIN)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
