"""Node, patch and Dirichlet bookkeeping on uniform Cartesian meshes (oracle).

Nodes are numbered lexicographically with x fastest; unknowns are interleaved
per node (dof = node * n_c + component), the node-blocked layout of
Section 4.3.

Patches (Section 4.3, "larger patches ... 4 adjacent elements in 2d or 8 in
3d"): patch P_i is a block of 2^d cells; its degrees of freedom are all
components of the 3^d nodes of that block.  Patches tile the cells without
overlap and overlap in the nodes they share.
"""

from __future__ import annotations

import itertools

import numpy as np


def nodes_per_dir(cells) -> tuple:
    return tuple(int(c) + 1 for c in cells)


def num_nodes(cells) -> int:
    return int(np.prod(nodes_per_dir(cells)))


def node_coords(cells) -> np.ndarray:
    """Integer node coordinates, shape (nodes, d), in node-number order."""
    nn = nodes_per_dir(cells)
    d = len(nn)
    grids = np.meshgrid(*[np.arange(n) for n in reversed(nn)], indexing="ij")
    return np.stack([grids[d - 1 - m].reshape(-1) for m in range(d)], axis=1)


def node_number(coords, cells) -> np.ndarray:
    nn = nodes_per_dir(cells)
    coords = np.asarray(coords)
    out = np.zeros(coords.shape[:-1], dtype=np.int64)
    stride = 1
    for m in range(len(nn)):
        out += coords[..., m] * stride
        stride *= nn[m]
    return out


def patch_nodes(cells) -> np.ndarray:
    """Node numbers of every patch, shape (patches, 3^d).

    Patch order: by patch origin (2 p_x, 2 p_y[, 2 p_z]) with p_x fastest;
    local node order: lexicographic offsets in {0,1,2}^d with x fastest.
    """
    d = len(cells)
    for c in cells:
        if c % 2:
            raise ValueError("Vanka patches of 2^d cells need an even cell count per direction")
    npd = [c // 2 for c in cells]
    origins = np.array([tuple(reversed(t)) for t in itertools.product(*[range(n) for n in reversed(npd)])],
                       dtype=np.int64) * 2                       # (patches, d), x fastest
    local = np.array([tuple(reversed(t)) for t in itertools.product(*[range(3)] * d)], dtype=np.int64)
    coords = origins[:, None, :] + local[None, :, :]
    return node_number(coords, cells)


def patch_dofs(cells, ncomp: int) -> np.ndarray:
    """Global unknown indices of every patch, shape (patches, 3^d * n_c), node-major."""
    nodes = patch_nodes(cells)
    return (nodes[:, :, None] * ncomp + np.arange(ncomp)[None, None, :]).reshape(nodes.shape[0], -1)


def coarse_mask(fine_mask: np.ndarray, fine_cells, ncomp: int) -> np.ndarray:
    """Dirichlet mask of the next coarser level by injection: coarse node I sits at fine node 2I."""
    coarse_cells = tuple(c // 2 for c in fine_cells)
    cc = node_coords(coarse_cells)
    fine_nodes = node_number(2 * cc, fine_cells)
    fm = np.asarray(fine_mask).reshape(-1, ncomp)
    return fm[fine_nodes].reshape(-1).astype(bool)


# ----------------------------------------------------------------------------
# Patches of two sizes (Section 5.5.1: small patches in the fluid, large ones
# in the solid).  A small patch is a block of 2^d cells (3^d nodes), a large
# one a block of 4^d cells (5^d nodes, the paper's four or eight adjacent
# elements).  Large patches sit on 4-aligned blocks whose cells are all
# flagged; every other cell belongs to the small patch of its 2-aligned block.
# ----------------------------------------------------------------------------

def coarse_cell_mask(fine_mask: np.ndarray) -> np.ndarray:
    """A coarse cell is flagged iff all its 2^d children are (array order
    reversed: (z,) y, x)."""
    m = np.asarray(fine_mask, dtype=bool)
    out = m
    for ax in range(m.ndim):
        n = out.shape[ax]
        if n % 2:
            raise ValueError("cell counts must be even to coarsen")
        a = np.take(out, np.arange(0, n, 2), axis=ax)
        b = np.take(out, np.arange(1, n, 2), axis=ax)
        out = a & b
    return out


def patch_blocks(cells, large_mask=None):
    """Patches as (origin, size) with origin the lowest cell (x, y[, z]) and
    size 2 or 4 cells per direction.  large_mask: None (small patches only) or
    bool per cell in array order ((z,) y, x).  Small patches come first in
    origin order (x fastest), then the large ones in origin order."""
    d = len(cells)
    for c in cells:
        if c % 2:
            raise ValueError("Vanka patches need an even cell count per direction")
    big = set()
    if large_mask is not None:
        m = np.asarray(large_mask, dtype=bool)
        if m.shape != tuple(reversed(cells)):
            raise ValueError("large_mask must have one entry per cell, array order (z, y, x)")
        starts = [range(0, c - 3, 4) for c in cells]
        for o in itertools.product(*reversed(starts)):      # o in array order
            sl = tuple(slice(v, v + 4) for v in o)
            if m[sl].all():
                big.add(tuple(reversed(o)))                  # (x, y[, z])
    small = []
    for o in itertools.product(*[range(0, c, 2) for c in reversed(cells)]):
        org = tuple(reversed(o))
        if tuple((v // 4) * 4 for v in org) not in big:
            small.append((org, 2))
    return small + [(org, 4) for org in sorted(big, key=lambda t: tuple(reversed(t)))]


def block_nodes(cells, origin, size) -> np.ndarray:
    """Node numbers of a (size+1)^d block of nodes at origin, lexicographic x fastest."""
    d = len(cells)
    local = np.array([tuple(reversed(t)) for t in itertools.product(*[range(size + 1)] * d)], dtype=np.int64)
    return node_number(np.asarray(origin, dtype=np.int64)[None, :] + local, cells)


def block_dofs(cells, ncomp: int, origin, size) -> np.ndarray:
    nodes = block_nodes(cells, origin, size)
    return (nodes[:, None] * ncomp + np.arange(ncomp)[None, :]).reshape(-1)
