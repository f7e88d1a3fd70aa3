"""The oracle reproduces the accuracy statements of the paper's Sections 4.2
and 4.3 over the full 28 x 28 x 2 grid of Experiment II (see exp2_grid)."""
import numpy as np

import oracle
from exp2_grid import check_paper_claims, problems


def test_oracle_follows_sections_4_2_and_4_3():
    rows = []
    for case, la, lz, A, Z in problems():
        loss = {}
        for v in ("naive", "ha", "hp"):
            Q, R, info, _, _ = oracle.mgs(A, Z, v, "row")
            loss[v] = oracle.orth_loss(A, Q) if info == 0 else np.inf
        rows.append((case, la, lz, loss))
    summary = check_paper_claims(rows)
    print(summary)
