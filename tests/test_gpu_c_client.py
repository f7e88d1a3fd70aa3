"""The plain-C client (tests/c/qr_tridiag.c) on the GPU: every form runs
through the C ABI from C, meets the invariants checked in C, and its R
matches the oracle's."""
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_c_client(tmp_path, variant):
    from c_client import build_client

    exe = build_client(str(tmp_path))
    m, n = 3000, 6
    rfile = os.path.join(str(tmp_path), "R.txt")
    r = subprocess.run([exe, str(m), str(n), str(variant), rfile], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.stdout, r.stderr)
    R = np.loadtxt(rfile).reshape(n, n).T
    A = W.tridiag_csr(m)
    k = np.arange(m)[:, None] + 1.0
    j = np.arange(n)[None, :] + 1.0
    Z = np.asfortranarray(np.sin(0.37 * k * j) + 0.01 * (j - 1))
    fn = oracle.cgs if variant >= 3 else oracle.mgs
    form = ["naive", "ha", "hp"][variant % 3]
    _, Ro, info, _, _ = fn(A, Z, form, "col")
    assert info == 0
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-10
