"""Build the CPU oracle (test infrastructure) into oracle/liboracle.so with plain g++."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")


FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"]


def compile_to(src_dir: str, out: str) -> None:
    """Compile oracle.cpp of src_dir (with its headers) into the shared library out."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["g++"] + FLAGS + [os.path.join(src_dir, "oracle.cpp"), "-o", tmp])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "oracle.cpp")
    deps = [src] + [os.path.join(HERE, h) for h in ("oracle.h", "dual.h", "counted.h")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
        return LIB
    compile_to(HERE, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
