"""Compile the CPU oracle (test infrastructure) into oracle/_liboracle.so.

Flags: -O2 -ffp-contract=off (no fused multiply-add unless the source calls
fmaf), -fPIC -shared, OpenMP when the compiler supports it (the per-particle
loops are independent, so the thread count never changes a result).  On
x86-64 hosts whose CPU has FMA, -mfma only makes fmaf a single instruction;
fmaf is correctly rounded either way, so results are identical.
"""
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "abc_oracle.c")
LIB = os.path.join(HERE, "_liboracle.so")


def _has_x86_fma() -> bool:
    if platform.machine() not in ("x86_64", "AMD64"):
        return False
    try:
        with open("/proc/cpuinfo") as f:
            return " fma " in f.read()
    except OSError:
        return False


def build_oracle(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11"]
    if _has_x86_fma():
        base.append("-mfma")
    tmp = LIB + ".tmp%d" % os.getpid()
    for extra in (["-fopenmp"], []):
        cmd = base + extra + [SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build_oracle(force=True))
