"""Compile the FP64 CPU oracle (plain C) into oracle/_build/liboracle.so, and the
all-core CPU baseline (OpenMP) into oracle/_build/libcpu_parallel.so.

Test infrastructure: the solver library never links or loads either.
``-ffp-contract=off`` keeps every FP32 operation of the successor rule a single
IEEE operation (no fused multiply-add), as that rule prescribes.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")
PAR_SRC = os.path.join(HERE, "cpu_parallel.c")
PAR_OUT = os.path.join(OUT_DIR, "libcpu_parallel.so")


def _fresh(out: str, src: str) -> bool:
    return os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src)


def _compile(cmd, out: str) -> None:
    # a per-process temporary name: concurrent builds never rename each other's file
    tmp = f"{out}.{os.getpid()}.tmp"
    subprocess.run(cmd + ["-o", tmp], check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not _fresh(OUT, SRC):
        _compile(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                  "-fPIC", "-shared", SRC, "-lm"], OUT)
    return OUT


def build_parallel(force: bool = False) -> str:
    """The all-core baseline; without OpenMP support it builds single-threaded."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not _fresh(PAR_OUT, PAR_SRC):
        base = ["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-fPIC", "-shared", PAR_SRC, "-lm"]
        try:
            _compile(base[:1] + ["-fopenmp"] + base[1:], PAR_OUT)
        except subprocess.CalledProcessError:
            _compile(base, PAR_OUT)
    return PAR_OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_parallel(force="--force" in sys.argv))
