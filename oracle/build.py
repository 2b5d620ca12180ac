"""Build the oracle's C helper (test infrastructure only): gcc -O2 -fopenmp -shared."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle_kron.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "kron_hv.c")
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    tmp = f"{LIB}.{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
