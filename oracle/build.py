"""TEST INFRASTRUCTURE ONLY: compiles the CPU oracle (plain g++, FP64, no FMA contraction).

liboracle.so        -- OpenMP over k-planes, used by tests and the CPU baseline
liboracle_count.so  -- single-threaded operation-counting build (-DORC_COUNTING)
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "orc.cpp")


def lib_path(counting=False):
    return os.path.join(HERE, "liboracle_count.so" if counting else "liboracle.so")


def build_oracle(force=False):
    deps = [SRC, os.path.join(HERE, "orc.h"), os.path.join(HERE, "counting.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    base = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-Wall", "-Wno-unknown-pragmas", SRC]
    for counting in (False, True):
        out = lib_path(counting)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        flags = ["-DORC_COUNTING"] if counting else ["-fopenmp"]
        tmp = out + ".tmp"
        subprocess.check_call(base + flags + ["-o", tmp])
        os.replace(tmp, out)
    return lib_path(False)


if __name__ == "__main__":
    print(build_oracle(force=True))
