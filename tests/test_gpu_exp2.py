"""The CUDA path follows the accuracy statements of Sections 4.2 and 4.3.

The whole 28 x 28 x 2 grid of Experiment II runs through mgsa_qr_batched
(1568 instances per variant, one call each); the losses of A-orthogonality
are evaluated on the host in double-double.  The same statements the
oracle satisfies (exp2_grid.check_paper_claims) must hold for the GPU
results.  Problem by problem, where the loss is at rounding level
(delta_1 <= 1e-10) the GPU's is within 10x the oracle's; where rounding errors
are amplified by the conditioning (the regime Section 3 bounds), two valid
rounding sequences legitimately differ more, and the GPU's loss must obey the
variant's bound (10 delta_1 for naive and HP, 10 delta_2 for HA, as the
oracle does) and stay within 100x the oracle's.
"""
import numpy as np
import pytest

import oracle
from exp2_grid import check_paper_claims, delta1, delta2, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402
from paper_1703_10440_gb300.batch import Batch  # noqa: E402


def test_gpu_follows_sections_4_2_and_4_3():
    probs = problems()
    inst = [(A, Z) for _, _, _, A, Z in probs]
    gpu = {}
    with mgsa.Handle(0) as h:
        for v in ("naive", "ha", "hp"):
            b = Batch(inst, v)
            b.run(h.h)
            torch.cuda.synchronize()
            out = []
            for k in range(b.count):
                Q, R, info = b.result(k)
                out.append(oracle.orth_loss(inst[k][0], Q) if info == 0 else np.inf)
            gpu[v] = out
    rows = [(c, la, lz, {v: gpu[v][k] for v in gpu}) for k, (c, la, lz, _, _) in enumerate(probs)]
    summary = check_paper_claims(rows)
    print(summary)
    ratios_well, ratios_ill = [], []
    for k, (c, la, lz, A, Z) in enumerate(probs):
        for v in ("naive", "ha", "hp"):
            Qo, _, info, _, _ = oracle.mgs(A, Z, v, "row")
            if info != 0:
                continue
            lo = oracle.orth_loss(A, Qo)
            g = gpu[v][k]
            d1 = delta1(la, lz)
            if d1 <= 1e-10:
                assert g <= max(1e-12, 10 * lo), (c, la, lz, v, g, lo)
                ratios_well.append(g / max(lo, 1e-16))
            elif lo <= 1e-8:
                bound = 10 * (delta2(la, lz) if v == "ha" else d1)
                assert g <= bound, (c, la, lz, v, g, bound)
                assert g <= 100 * lo, (c, la, lz, v, g, lo)
                ratios_ill.append(g / lo)
    print("gpu/oracle loss, delta1 <= 1e-10: median %.3g max %.3g (%d)" %
          (np.median(ratios_well), np.max(ratios_well), len(ratios_well)))
    print("gpu/oracle loss, ill-conditioned: median %.3g max %.3g (%d)" %
          (np.median(ratios_ill), np.max(ratios_ill), len(ratios_ill)))
