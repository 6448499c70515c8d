"""Compile the C oracle into oracle/liboracle_hisq.so with the system C compiler.

Test infrastructure: the oracle is the checker for the CUDA library, never part of it.
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "hisq_oracle.c")
LIBRARY = os.path.join(HERE, "liboracle_hisq.so")
LIBRARY_OMP = os.path.join(HERE, "liboracle_hisq_omp.so")  # the same code, site loops on all cores


def build(force: bool = False, output: str = LIBRARY, source: str = SOURCE, openmp: bool = False) -> str:
    """Build the oracle library (skipped when up to date) and return its path."""
    stamp = output + ".machine"
    same_machine = os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()
    if (not force and same_machine and os.path.exists(output)
            and os.path.getmtime(output) >= os.path.getmtime(source)):
        return output
    cc = os.environ.get("CC", "gcc")
    cmd = [cc, "-O2", "-std=c99", "-Wall", "-Wno-unknown-pragmas", "-shared", "-fPIC"]
    cmd += ["-fopenmp"] if openmp else []
    cmd += ["-o", output, source, "-lm"]
    subprocess.run(cmd, check=True)
    with open(stamp, "w") as f:
        f.write(platform.machine())
    return output


def build_all(force: bool = False) -> None:
    """The single-threaded oracle (tests, parity) and its OpenMP build (all-core CPU baseline)."""
    build(force)
    build(force, output=LIBRARY_OMP, openmp=True)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
    print(LIBRARY, LIBRARY_OMP)
