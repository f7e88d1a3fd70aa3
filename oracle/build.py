"""Build the CPU oracle shared library (test infrastructure only).

The oracle is plain C compiled with gcc.  ``-ffp-contract=off`` keeps every
``a*b + c`` as two rounded operations (gcc contracts to FMA by default on
aarch64), so the oracle computes exactly the expressions it spells out on
both x86_64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mgs_oracle.c")
PAR_SRC = os.path.join(HERE, "mgs_oracle_par.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmgsa_oracle.so")
PAR_LIB = os.path.join(OUT_DIR, "libmgsa_oracle_par.so")

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall"]


def build(force: bool = False, extra_flags: list[str] | None = None, out: str | None = None) -> str:
    """Compile ``mgs_oracle.c`` and return the path of the shared library.

    ``extra_flags``/``out`` let a test compile a variant of the oracle (for
    example one with a planted mistake) into a separate library.
    """
    out = out or LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    stamp = out + ".host_arch"
    if not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine():
        force = True
    if not force and extra_flags is None and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    cmd = ["gcc", *CFLAGS, *(extra_flags or []), "-o", out + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    with open(stamp, "w") as f:
        f.write(platform.machine())
    return out


def build_par(force: bool = False) -> str:
    """Compile ``mgs_oracle_par.c`` (the multi-core build of the row-oriented
    algorithms) with OpenMP; without a working ``-fopenmp`` it is compiled
    without it and runs on one thread."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = PAR_LIB + ".host_arch"
    if not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine():
        force = True
    if not force and os.path.exists(PAR_LIB) and os.path.getmtime(PAR_LIB) >= os.path.getmtime(PAR_SRC):
        return PAR_LIB
    base = ["gcc", *CFLAGS, "-o", PAR_LIB + ".tmp", PAR_SRC, "-lm"]
    if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(PAR_LIB + ".tmp", PAR_LIB)
    with open(stamp, "w") as f:
        f.write(platform.machine())
    return PAR_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_par(force="--force" in sys.argv))
