"""The C-ABI library loads and exports every entry point include/*.h declares.

No compute is launched here: these run without a GPU.  Argument checks that
happen before any CUDA call (NULL handle / pointers) are exercised too.
"""
import ctypes
import glob
import os
import re

import pytest

from paper_1703_10440_gb300 import mgsa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(mgsa_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mgsa_create", "mgsa_qr", "mgsa_get_info", "mgsa_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(mgsa.lib()._name)  # a fresh handle, without the binding's signatures
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(mgsa.SIGNATURES) == declared_functions()


def test_host_side_argument_errors():
    lib = mgsa.lib()
    A = mgsa.mgsa_csr(4, 4, None, None, None)
    st = lib.mgsa_qr(None, ctypes.byref(A), None, 4, 2, 4, 0, None, 4, None, 2, None)
    assert st == mgsa.MGSA_ERR_INVALID
    info = ctypes.c_int(0)
    assert lib.mgsa_get_info(None, None, ctypes.byref(info)) == mgsa.MGSA_ERR_INVALID
    assert lib.mgsa_create(None, 0) == mgsa.MGSA_ERR_INVALID
    assert lib.mgsa_destroy(None) == mgsa.MGSA_OK
    assert isinstance(mgsa.mgsa_last_error(), str)


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = mgsa.lib().mgsa_create(ctypes.byref(h), 0)
    assert st in (mgsa.MGSA_ERR_CUDA, mgsa.MGSA_ERR_INVALID)
    assert h.value is None


def test_plain_c_client_builds_and_fails_cleanly_without_gpu(tmp_path):
    """include/mgsa.h is a C11 header: a C program compiles against it with
    -Wall -Wextra -Werror -pedantic, links libmgsa, and (without a GPU)
    mgsa_create reports an error instead of crashing."""
    import subprocess

    import torch
    from c_client import build_client

    exe = build_client(str(tmp_path))
    if torch.cuda.is_available():
        return  # the GPU run is tests/test_gpu_c_client.py
    r = subprocess.run([exe, "100", "4", "1"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.startswith("nogpu"), (r.stdout, r.stderr)


def header_constants():
    """Enumerators (NAME = integer) and integer #defines of include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for name, val in re.findall(r"\b(MGSA_\w+)\s*=\s*(-?\d+)\s*[,}]", text):
            out[name] = int(val)
        for name, val in re.findall(r"^#define\s+(MGSA_\w+)\s+\(?(-?\d+)\)?\s*$", text, flags=re.M):
            out[name] = int(val)
        for name, val, sh in re.findall(r"^#define\s+(MGSA_\w+)\s+\((\d+)u\s*<<\s*(\d+)\)", text, flags=re.M):
            out[name] = int(val) << int(sh)
    return out


def test_binding_constants_match_the_header():
    consts = header_constants()
    for name in ("MGSA_NAIVE", "MGSA_CGS_HP", "MGSA_ERR_TIMEOUT", "MGSA_PARAM_WAIT_FAULT", "MGSA_MAX_N",
                 "MGSA_BATCH_MAX_N", "MGSA_NOALLOC_SCRATCH_BYTES"):
        assert name in consts, name
    for name, val in consts.items():
        if hasattr(mgsa, name):
            assert getattr(mgsa, name) == val, (name, getattr(mgsa, name), val)
    missing = sorted(n for n in consts if not hasattr(mgsa, n))
    assert not missing, missing
