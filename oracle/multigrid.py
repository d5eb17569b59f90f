"""Geometric multigrid V-cycle preconditioner, item (II) of Section 4.3 (oracle).

Each level carries its own assembled matrix (rediscretisation, as in
Section 5.5.2).  One application z = M^{-1} r of the V(nu1, nu2) cycle, from
a zero initial guess on every level:

    level l > 0:  nu1 Vanka steps (Eq. (vanka)) on A_l x = b
                  r = b - A_l x;  b_{l-1} = P^T r, Dirichlet entries set to 0
                  x_{l-1} = V-cycle on level l-1
                  x += P x_{l-1}, Dirichlet entries of the correction set to 0
                  nu2 Vanka steps
    level 0:      exact solve with a dense LU factorisation (partial pivoting)

Readings where the paper is silent: Q1 interpolation transfers (see
``transfer``), a direct coarsest-level solve, Vanka on every level above the
coarsest, and the overlap weighting of the Vanka sum (see ``vanka``).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .bsr import BlockMatrix
from .mesh import coarse_cell_mask, coarse_mask, patch_dofs
from .transfer import prolongation
from .vanka import (group_weights, overlap_weights, patch_groups, patch_inverses, patch_matrices, vanka_step,
                    vanka_step_groups)


class Level:
    def __init__(self, cells, row_ptr, col_idx, vals, mask, smooth: bool, weighting: str, large_mask=None):
        self.cells = tuple(int(c) for c in cells)
        self.A = BlockMatrix(row_ptr, col_idx, vals)
        self.ncomp = self.A.ncomp
        self.mask = np.asarray(mask, dtype=bool)
        self.P = None            # prolongation from the next coarser level
        self.dofs = None
        self.Ainv = None
        self.weight = None
        self.groups = None       # patches of two sizes: [(dofs, inverses)] per size
        if smooth and large_mask is not None and np.asarray(large_mask).any():
            self.groups = patch_groups(self.A, self.cells, large_mask)
            self.weight = group_weights(self.groups, self.A.size, weighting)
            if len(self.groups) == 1:    # no 4-aligned block fits the region on this level
                self.dofs, self.Ainv = self.groups[0]
                self.groups = None
        elif smooth:
            self.dofs = patch_dofs(self.cells, self.ncomp)
            self.Ainv = patch_inverses(patch_matrices(self.A, self.cells))
            self.weight = overlap_weights(self.dofs, self.A.size, weighting)


class Hierarchy:
    """Levels coarsest first; ``levels`` holds objects with cells/row_ptr/col_idx/vals."""

    def __init__(self, levels, fine_mask, nu1=2, nu2=2, omega=0.8, weighting="average", large_cells=None):
        """large_cells: None, or bool per finest-level cell (array order (z,) y, x)
        flagging the region of large patches (Section 5.5.1); a coarse cell is
        flagged iff all its children are."""
        self.nu1, self.nu2, self.omega = int(nu1), int(nu2), float(omega)
        L = len(levels)
        masks = [None] * L
        masks[L - 1] = np.asarray(fine_mask, dtype=bool)
        nc = levels[-1].vals.shape[1]
        for lev in range(L - 1, 0, -1):
            for a, b in zip(levels[lev].cells, levels[lev - 1].cells):
                if a != 2 * b:
                    raise ValueError("levels must halve the cell count per direction")
            masks[lev - 1] = coarse_mask(masks[lev], levels[lev].cells, nc)
        large = [None] * L
        if large_cells is not None:
            large[L - 1] = np.asarray(large_cells, dtype=bool)
            for lev in range(L - 1, 0, -1):
                large[lev - 1] = coarse_cell_mask(large[lev])
        self.levels = []
        for lev, m in enumerate(levels):
            self.levels.append(Level(m.cells, m.row_ptr, m.col_idx, m.vals, masks[lev], smooth=lev > 0,
                                     weighting=weighting, large_mask=large[lev]))
        for lev in range(1, L):
            self.levels[lev].P = prolongation(self.levels[lev - 1].cells, nc)
        self.coarse_lu = sla.lu_factor(self.levels[0].A.dense())

    @property
    def fine(self) -> Level:
        return self.levels[-1]

    def smooth(self, lev: int, b, x, steps: int):
        L = self.levels[lev]
        for _ in range(steps):
            if L.groups is not None:
                x = vanka_step_groups(L.A, L.groups, b, x, self.omega, L.weight)
            else:
                x = vanka_step(L.A, L.Ainv, L.dofs, b, x, self.omega, L.weight)
        return x

    def restrict_residual(self, lev: int, b, x):
        L = self.levels[lev]
        r = b - L.A.matvec(x)
        rc = L.P.T @ r
        rc[self.levels[lev - 1].mask] = 0.0
        return rc

    def prolongate(self, lev: int, ec):
        L = self.levels[lev]
        c = L.P @ ec
        c[L.mask] = 0.0
        return c

    def coarse_solve(self, b):
        return sla.lu_solve(self.coarse_lu, b)

    def vcycle(self, b, lev: int = None):
        if lev is None:
            lev = len(self.levels) - 1
        if lev == 0:
            return self.coarse_solve(b)
        x = np.zeros_like(b)
        x = self.smooth(lev, b, x, self.nu1)
        rc = self.restrict_residual(lev, b, x)
        ec = self.vcycle(rc, lev - 1)
        x = x + self.prolongate(lev, ec)
        x = self.smooth(lev, b, x, self.nu2)
        return x
