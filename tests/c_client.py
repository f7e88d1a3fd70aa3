"""Build the plain-C clients of libmgsa (tests/c/*.c) with gcc."""
import os
import subprocess

from paper_1703_10440_gb300 import build as lib_build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def build_client(out_dir: str, name: str = "qr_tridiag") -> str:
    lib = lib_build.LIB if os.path.exists(lib_build.LIB) else lib_build.build()
    exe = os.path.join(out_dir, name)
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(HERE, "c", name + ".c"), "-o", exe,
           lib, "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm",
           "-Wl,-rpath," + os.path.dirname(lib), "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe
