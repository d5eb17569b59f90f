"""Grid transfers between nested uniform levels (oracle side).

The paper names a geometric V-cycle on nested meshes but not its transfers.
The reading used here: prolongation P is Q1 nodal interpolation (coarse
node I sits at fine node 2I; a fine node at an odd position averages its two
coarse neighbours in that direction, tensorised over directions) applied to
every component; restriction is its transpose P^T.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def interpolation_1d(coarse_cells: int) -> sp.csr_matrix:
    nf = 2 * coarse_cells + 1
    ncn = coarse_cells + 1
    rows, cols, vals = [], [], []
    for i in range(nf):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, ncn))


def prolongation(coarse_cells, ncomp: int) -> sp.csr_matrix:
    """P from the coarse level (cells per direction) to the level twice as fine."""
    P = None
    for c in coarse_cells:                   # x first; the slower index goes left in kron
        p1 = interpolation_1d(int(c))
        P = p1 if P is None else sp.kron(p1, P, format="csr")
    return sp.kron(P, sp.identity(ncomp, format="csr"), format="csr")
