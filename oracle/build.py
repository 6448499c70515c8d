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


def build(force: bool = False, output: str = LIBRARY, source: str = SOURCE) -> str:
    """Build the oracle library (skipped when up to date) and return its path."""
    stamp = output + ".machine"
    same_machine = os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()
    if (not force and same_machine and os.path.exists(output)
            and os.path.getmtime(output) >= os.path.getmtime(source)):
        return output
    cc = os.environ.get("CC", "gcc")
    cmd = [cc, "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", "-o", output, source, "-lm"]
    subprocess.run(cmd, check=True)
    with open(stamp, "w") as f:
        f.write(platform.machine())
    return output


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
