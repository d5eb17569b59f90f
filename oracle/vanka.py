"""Vanka patch smoother, Eq. (vanka) of Section 4.3 (oracle side).

    d = b - A x
    x <- x + omega_V * sum_i R_i^T A_i^{-1} R_i d,     A_i = R_i A R_i^T

The patches are combined additively ("Jacobi coupling").  Reading of the
sum: as printed, every patch correction is added in full; with patches of
2^d cells every mesh vertex lies in up to 2^d patches, and the printed sum
with omega_V = 0.8 then diverges on these operators (error growth of about
2.5x per step on the 2d workloads).  The default reading keeps the paper's
omega_V = 0.8 and weights each unknown's summed correction by 1 / m, m the
number of patches that contain it (a partition of unity over the overlap);
``weighting="sum"`` gives the printed plain sum.  The local matrices are
inverted exactly (LAPACK getrf/getri through numpy.linalg.inv, i.e. LU with
partial pivoting).
"""

from __future__ import annotations

import numpy as np

from .mesh import block_nodes, patch_blocks, patch_nodes


def patch_matrices(A, cells) -> np.ndarray:
    """A_i = R_i A R_i^T for every patch, shape (patches, n_p, n_p), n_p = 3^d n_c."""
    return node_block_matrices(A, patch_nodes(cells))


def node_block_matrices(A, nodes) -> np.ndarray:
    """R_i A R_i^T for patches given by their node lists nodes (P, m):
    shape (P, m n_c, m n_c), unknowns node-major."""
    P, m = nodes.shape
    nc = A.ncomp
    blocks = A.block_lookup(nodes[:, :, None], nodes[:, None, :])   # (P, m, m, nc, nc)
    return blocks.transpose(0, 1, 3, 2, 4).reshape(P, m * nc, m * nc)


def patch_inverses(Ap: np.ndarray) -> np.ndarray:
    """Exact inverses of the patch matrices (Section 4.3: "inverted exactly")."""
    return np.linalg.inv(Ap)


def overlap_weights(dofs, size: int, weighting: str = "average") -> np.ndarray:
    """Per-unknown weight of the summed patch corrections: 1/m ("average") or 1 ("sum")."""
    if weighting == "sum":
        return np.ones(size)
    if weighting != "average":
        raise ValueError(weighting)
    m = np.zeros(size)
    np.add.at(m, dofs, 1.0)
    return 1.0 / m


def vanka_step(A, Ainv, dofs, b, x, omega, weight):
    """One additive Vanka iteration of Eq. (vanka) with overlap weights ``weight``."""
    d = b - A.matvec(x)
    local = np.einsum("pij,pj->pi", Ainv, d[dofs])
    corr = np.zeros_like(x)
    np.add.at(corr, dofs, local)
    return x + omega * weight * corr


def patch_groups(A, cells, large_mask=None):
    """The patches of a level with their exact inverses, grouped by size:
    a list of (dofs (P, n_p), inverses (P, n_p, n_p)), small patches (2^d
    cells) first, then large ones (4^d cells) where large_mask flags whole
    4-aligned blocks (mesh.patch_blocks)."""
    nc = A.ncomp
    out = []
    blocks = patch_blocks(cells, large_mask)
    for size in (2, 4):
        sel = [o for o, s in blocks if s == size]
        if not sel:
            continue
        nodes = np.stack([block_nodes(cells, o, size) for o in sel])
        dofs = (nodes[:, :, None] * nc + np.arange(nc)[None, None, :]).reshape(nodes.shape[0], -1)
        out.append((dofs, patch_inverses(node_block_matrices(A, nodes))))
    return out


def group_weights(groups, size: int, weighting: str = "average") -> np.ndarray:
    """overlap_weights over the patches of every group."""
    if weighting == "sum":
        return np.ones(size)
    if weighting != "average":
        raise ValueError(weighting)
    m = np.zeros(size)
    for dofs, _ in groups:
        np.add.at(m, dofs, 1.0)
    return 1.0 / m


def vanka_step_groups(A, groups, b, x, omega, weight):
    """Eq. (vanka) with patches of several sizes: the corrections of every
    patch of every group summed, then weighted and damped."""
    d = b - A.matvec(x)
    corr = np.zeros_like(x)
    for dofs, Ainv in groups:
        np.add.at(corr, dofs, np.einsum("pij,pj->pi", Ainv, d[dofs]))
    return x + omega * weight * corr
