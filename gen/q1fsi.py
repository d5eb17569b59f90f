"""Q1 assembly of the condensed momentum Jacobian on uniform Cartesian meshes.

The operator (Section 3, Eq. (aletime:2) with theta = 1, the condensation of
Eq. (defgrad) and the reduced Jacobian of Eq. (REDUCEDMATRIX)/(problem:1)) is
read as follows; every choice the paper leaves open is named here.

Unknowns per node: (v_1, .., v_d, p), interleaved per node (node-blocked
vectors of Section 4.3, block size n_c = d + 1).  Densities are 1 (the paper's
fluid and solid densities are equal, Section 5.1).

Fluid cells (test functions phi for velocity, xi for pressure):
    (dv, phi) + k nu (grad dv + grad dv^T, grad phi) + k ((b . grad) dv, phi)
    - k (dp, div phi)                                  [momentum rows]
    k (div dv, xi) + k alpha_h (grad dp, grad xi)      [divergence rows]
Solid cells (deformation condensed, so the elastic term is scaled by k^2:
k * [2 (k mu_s) (eps dv, eps phi) + (k lambda_s) (div dv, div phi)]):
    (dv, phi) + k [2 (k mu_s)(eps(dv), eps(phi)) + (k lambda_s)(div dv, div phi)]
    k alpha_f (grad dp, grad xi)                       [pressure extension only]
alpha_h = alpha h^2 / nu is the equal-order (Brezzi-Pitkaranta) pressure
stabilisation with the usual h^2/nu scaling; it replaces the paper's Q2
local-projection stabilisation.  The pressure acts in the fluid and on the
interface only (Section 3.2), so solid cells carry no pressure-velocity
coupling; their pressure unknowns are a harmonic extension with the fixed
coefficient alpha_f = alpha h_fine^2 / nu of the finest level, which keeps
that extension the same operator on every level (a rediscretised h^2 there
makes each coarse level 2^d times too stiff and the multigrid iteration
counts then grow with the number of levels).  Quadrature is the 2^d-point
Gauss rule per cell.  Homogeneous Dirichlet conditions on every velocity
component on the boundary (optionally except outflow faces, left natural):
row and column zeroed, diagonal 1.

Every multigrid level is rediscretised (Section 5.5.2: matrices are assembled
on every level).  Item (II) of Section 4.3 asks every level to resolve the
fluid-solid interface, so a cell is solid iff the centroid of its ancestor
on the coarsest level lies in the solid region: all levels then share the
interface of the coarsest mesh.

Storage: block sparse rows (BSR) over mesh nodes, n_c x n_c blocks stored
row-major, columns ascending within a row (Section 4.3's block matrices).
Nodes are numbered lexicographically with x fastest.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np


# ----------------------------------------------------------------------------
# problem description
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Coefficients:
    k: float = 0.01          # time-step size
    nu: float = 1e-2         # fluid kinematic viscosity
    kmu_s: float = 1e2       # k * mu_s  (condensed solid shear stiffness)
    klam_s: float = 4e2      # k * lambda_s
    alpha: float = 0.1       # pressure stabilisation alpha_h = alpha * h^2 / nu
    convection: bool = True  # Oseen convection term in fluid cells


@dataclass(frozen=True)
class Problem:
    dim: int
    n: tuple                                   # finest-level cells per direction (x, y[, z])
    levels: int
    solid: Optional[tuple] = None              # (axis, sign, threshold): solid iff sign*(c[axis]-thr) > 0
    conv_seed: int = 0
    rhs_seed: int = 1
    coef: Coefficients = field(default_factory=Coefficients)
    outflow: tuple = ()                        # faces (axis, side) left natural (do-nothing), side 0/1

    @property
    def ncomp(self) -> int:
        return self.dim + 1


def config_problem(name: str, **overrides) -> Problem:
    """The synthetic workloads the solver is measured on.

    cfg1: 2d 32x32, solid x > 0.6, 3 levels        (3,267 unknowns)
    cfg2: 2d 256x256, same coefficients, 7 levels  (198,147 unknowns)
    cfg3: 3d 32^3, solid z < 0.25, 4 levels        (143,748 unknowns)
    cfg4: 3d 96^3, 6 levels                        (3,650,692 unknowns)
    """
    table = {
        "cfg1": dict(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6)),
        "cfg2": dict(dim=2, n=(256, 256), levels=7, solid=(0, +1, 0.6)),
        "cfg3": dict(dim=3, n=(32, 32, 32), levels=4, solid=(2, -1, 0.25)),
        "cfg4": dict(dim=3, n=(96, 96, 96), levels=6, solid=(2, -1, 0.25)),
    }
    kw = dict(table[name])
    kw.update(overrides)
    return Problem(**kw)


def level_cells(problem: Problem) -> list:
    """Cells per direction on every level, coarsest first."""
    out = []
    for lev in range(problem.levels):
        f = 2 ** (problem.levels - 1 - lev)
        for nk in problem.n:
            if nk % f:
                raise ValueError(f"{problem.n} cells not divisible by 2^{problem.levels - 1}")
        out.append(tuple(nk // f for nk in problem.n))
    return out


# ----------------------------------------------------------------------------
# convection field: a seeded smooth random field with |b|_2 <= 1
# ----------------------------------------------------------------------------

class ConvectionField:
    """b_c(x) = s * sum_m a_{c,m} sin(2 pi kappa_m . x + phi_{c,m}).

    kappa_m in {0,1,2}^d, a ~ U[-1,1], phi ~ U[0, 2 pi), drawn in that order
    from numpy's default_rng(seed).  s = 1 / sum_m ||a_{:,m}||_2, which bounds
    |b(x)|_2 <= 1 everywhere (triangle inequality) and does not depend on the
    mesh, so every level sees the same continuous field.
    """

    def __init__(self, dim: int, seed: int, modes: int = 4):
        rng = np.random.default_rng(seed)
        self.dim = dim
        self.kappa = rng.integers(0, 3, size=(modes, dim)).astype(np.float64)
        self.amp = rng.uniform(-1.0, 1.0, size=(dim, modes))
        self.phase = rng.uniform(0.0, 2.0 * np.pi, size=(dim, modes))
        self.scale = 1.0 / float(np.sum(np.linalg.norm(self.amp, axis=0)))

    def __call__(self, x: np.ndarray) -> np.ndarray:
        arg = 2.0 * np.pi * (x @ self.kappa.T)            # (..., modes)
        out = np.empty(x.shape[:-1] + (self.dim,))
        for c in range(self.dim):
            out[..., c] = self.scale * np.sum(self.amp[c] * np.sin(arg + self.phase[c]), axis=-1)
        return out


# ----------------------------------------------------------------------------
# reference Q1 element on [0,1]^d
# ----------------------------------------------------------------------------

def reference_element(dim: int):
    """Q1 shape functions at the 2^d Gauss points of [0,1]^d.

    Local node a has position bits (a & 1, a >> 1 & 1, a >> 2 & 1) (x fastest);
    quadrature points are ordered the same way.  Returns
    (xi[q, d], w[q], psi[q, a], dpsi[q, a, m]) with derivatives in xi.
    """
    g = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))
    nq = na = 2 ** dim
    xi = np.array([[g[(q >> m) & 1] for m in range(dim)] for q in range(nq)])
    w = np.full(nq, 1.0 / nq)
    psi = np.ones((nq, na))
    dpsi = np.ones((nq, na, dim))
    for a in range(na):
        bits = [(a >> m) & 1 for m in range(dim)]
        for m in range(dim):
            f = xi[:, m] if bits[m] else 1.0 - xi[:, m]
            df = 1.0 if bits[m] else -1.0
            psi[:, a] *= f
            for mm in range(dim):
                dpsi[:, a, mm] *= df if mm == m else f
    return xi, w, psi, dpsi


def _element_blocks(dim: int, h: float, coef: Coefficients, h_fine: float):
    """Constant parts of the fluid and solid element matrices, E[a, i, b, j].

    h is this level's cell size, h_fine the finest level's (used by the
    solid-cell pressure term, which is the same on every level).
    """
    _, w, psi, dpsi = reference_element(dim)
    nc = dim + 1
    na = 2 ** dim
    M = h ** dim * np.einsum("q,qa,qb->ab", w, psi, psi)
    G = h ** (dim - 2) * np.einsum("q,qam,qbm->ab", w, dpsi, dpsi)
    D = h ** (dim - 2) * np.einsum("q,qam,qbn->abmn", w, dpsi, dpsi)   # int d_m psi_a d_n psi_b
    B = h ** (dim - 1) * np.einsum("q,qa,qbm->abm", w, psi, dpsi)      # int psi_a d_m psi_b
    k = coef.k
    alpha_h = coef.alpha * h * h / coef.nu
    Ef = np.zeros((na, nc, na, nc))
    Es = np.zeros((na, nc, na, nc))
    for i in range(dim):
        for j in range(dim):
            # viscous: k nu [delta_ij grad psi_a . grad psi_b + d_j psi_a d_i psi_b]
            Ef[:, i, :, j] = k * coef.nu * D[:, :, j, i]
            # condensed elasticity: k [kmu (delta_ij G + d_j psi_a d_i psi_b) + klam d_i psi_a d_j psi_b]
            Es[:, i, :, j] = k * coef.kmu_s * D[:, :, j, i] + k * coef.klam_s * D[:, :, i, j]
        Ef[:, i, :, i] += M + k * coef.nu * G
        Es[:, i, :, i] += M + k * coef.kmu_s * G
        Ef[:, i, :, dim] = -k * B[:, :, i].T          # -k (psi_b, d_i psi_a)
        Ef[:, dim, :, i] = k * B[:, :, i]             #  k (d_i psi_b, psi_a)
    Ef[:, dim, :, dim] = k * alpha_h * G
    Es[:, dim, :, dim] = k * (coef.alpha * h_fine * h_fine / coef.nu) * G
    return Ef, Es


def _convection_blocks(dim: int, cells: tuple, h: float, coef: Coefficients,
                       conv: Callable) -> np.ndarray:
    """k ((b . grad) psi_b, psi_a) per cell, shape cells_shape + (na, na)."""
    xi, w, psi, dpsi = reference_element(dim)
    shape = tuple(reversed(cells))                       # array order (z, y, x)
    axes = [np.arange(nk) * h for nk in cells]           # cell origins per direction
    origin = np.stack(np.meshgrid(*reversed(axes), indexing="ij")[::-1], axis=-1)  # shape + (d,)
    xq = origin[..., None, :] + h * xi                   # shape + (nq, d)
    bq = conv(xq)                                        # shape + (nq, d)
    bgrad = np.einsum("...qm,qbm->...qb", bq, dpsi)      # b . grad_xi psi_b at q
    return coef.k * h ** (dim - 1) * np.einsum("q,qa,...qb->...ab", w, psi, bgrad)


# ----------------------------------------------------------------------------
# assembly
# ----------------------------------------------------------------------------

@dataclass
class LevelMatrix:
    cells: tuple              # cells per direction (x, y[, z])
    row_ptr: np.ndarray       # int64, nodes + 1
    col_idx: np.ndarray       # int32, nnzb
    vals: np.ndarray          # float64, (nnzb, nc, nc), row-major blocks

    @property
    def nodes(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def ncomp(self) -> int:
        return int(self.vals.shape[1])


def _offsets(dim: int):
    """Stencil offsets o(s) in {-1,0,1}^d with s = sum_k (o_k + 1) 3^k."""
    return [tuple(((s // 3 ** m) % 3) - 1 for m in range(dim)) for s in range(3 ** dim)]


def _slices(pos, cells):
    """Array slice (z, y, x order) of the nodes cell + pos over all cells."""
    return tuple(slice(p, p + nk) for p, nk in zip(reversed(pos), reversed(cells)))


def solid_cells(problem: Problem, cells: tuple, coarse_cells: Optional[tuple] = None) -> np.ndarray:
    """Cell classification (array order z, y, x): solid iff the centroid of the
    cell's ancestor on the coarsest level lies in the solid region, so that
    every level resolves the same interface (item (II) of Section 4.3)."""
    h = 1.0 / cells[0]
    cshape = tuple(reversed(cells))
    if coarse_cells is None:
        coarse_cells = level_cells(problem)[0]
    r = cells[0] // coarse_cells[0]
    axes = [((np.arange(nk) // r) + 0.5) * r * h for nk in cells]
    cent = np.meshgrid(*reversed(axes), indexing="ij")[::-1]   # list over x, y, z
    if problem.solid is None:
        return np.zeros(cshape, dtype=bool)
    ax, sign, thr = problem.solid
    return sign * (cent[ax] - thr) > 0


def assemble_level(problem: Problem, cells: tuple, conv: Optional[Callable] = None,
                   solid_mask: Optional[np.ndarray] = None,
                   coarse_cells: Optional[tuple] = None) -> LevelMatrix:
    """Assemble the condensed-momentum Jacobian on one uniform level.

    The domain is [0, 1] in x with square cells of size h = 1 / cells[0]
    (other directions extend cells[k] * h).
    """
    dim = problem.dim
    nc = dim + 1
    na = 2 ** dim
    coef = problem.coef
    h = 1.0 / cells[0]
    nodes_n = tuple(nk + 1 for nk in cells)
    nshape = tuple(reversed(nodes_n))
    cshape = tuple(reversed(cells))
    nst = 3 ** dim

    if solid_mask is None:
        solid_mask = solid_cells(problem, cells, coarse_cells)
    fluid = (~solid_mask).astype(np.float64)
    solid = solid_mask.astype(np.float64)

    Ef, Es = _element_blocks(dim, h, coef, h_fine=1.0 / problem.n[0])
    Ec = None
    if coef.convection:
        if conv is None:
            conv = ConvectionField(dim, problem.conv_seed)
        Ec = _convection_blocks(dim, cells, h, coef, conv) * fluid[..., None, None]

    S = np.zeros(nshape + (nst, nc, nc))
    eye_v = np.zeros((nc, nc))
    eye_v[np.arange(dim), np.arange(dim)] = 1.0
    for a in range(na):
        pa = tuple((a >> m) & 1 for m in range(dim))
        rows = _slices(pa, cells)
        for b in range(na):
            pb = tuple((b >> m) & 1 for m in range(dim))
            s = sum((pb[m] - pa[m] + 1) * 3 ** m for m in range(dim))
            blk = fluid[..., None, None] * Ef[a, :, b, :] + solid[..., None, None] * Es[a, :, b, :]
            if Ec is not None:
                blk = blk + Ec[..., a, b][..., None, None] * eye_v
            S[rows + (s,)] += blk

    # homogeneous Dirichlet on velocity at boundary nodes: zero row and column, unit diagonal
    bnd = _dirichlet_nodes(dim, cells, problem.outflow)
    S[bnd, :, :dim, :] = 0.0
    offs = _offsets(dim)
    for s, o in enumerate(offs):
        # column node = row node + o; zero velocity columns where that node is on the boundary
        src = []
        dst = []
        for m in reversed(range(dim)):
            lo = max(0, -o[m])
            hi = nodes_n[m] - max(0, o[m])
            dst.append(slice(lo, hi))
            src.append(slice(lo + o[m], hi + o[m]))
        colb = np.zeros(nshape, dtype=bool)
        colb[tuple(dst)] = bnd[tuple(src)]
        sub = S[..., s, :, :dim]
        sub[colb] = 0.0
    center = (nst - 1) // 2
    for i in range(dim):
        S[..., center, i, i][bnd] = 1.0

    return _stencil_to_bsr(S, dim, cells, nc)


def _stencil_to_bsr(S: np.ndarray, dim: int, cells: tuple, nc: int) -> LevelMatrix:
    """BSR conversion of a node-stencil array S[nodes (z, y, x), s, nc, nc]:
    keep every in-range stencil block (the Q1 node-adjacency pattern)."""
    nodes_n = tuple(nk + 1 for nk in cells)
    nshape = tuple(reversed(nodes_n))
    nst = 3 ** dim
    offs = _offsets(dim)
    nodes = int(np.prod(nodes_n))
    valid = np.zeros(nshape + (nst,), dtype=bool)
    for s, o in enumerate(offs):
        sl = []
        for m in reversed(range(dim)):
            sl.append(slice(max(0, -o[m]), nodes_n[m] - max(0, o[m])))
        valid[tuple(sl) + (s,)] = True
    valid = valid.reshape(nodes, nst)
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(nodes + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    strides = [int(np.prod(nodes_n[:m])) for m in range(dim)]
    lin = np.array([sum(o[m] * strides[m] for m in range(dim)) for o in offs], dtype=np.int64)
    node_ids, s_ids = np.nonzero(valid)
    col_idx = (node_ids + lin[s_ids]).astype(np.int32)
    vals = S.reshape(nodes, nst, nc, nc)[valid]
    return LevelMatrix(cells=tuple(cells), row_ptr=row_ptr, col_idx=col_idx,
                       vals=np.ascontiguousarray(vals))


def _dirichlet_nodes(dim: int, cells: tuple, outflow=()) -> np.ndarray:
    """Boundary nodes carrying Dirichlet velocity (all faces except the outflow faces)."""
    nodes_n = tuple(nk + 1 for nk in cells)
    nshape = tuple(reversed(nodes_n))
    bnd = np.zeros(nshape, dtype=bool)
    for ax in range(dim):
        for side in (0, 1):
            if (ax, side) in tuple(tuple(f) for f in outflow):
                continue
            idx = [slice(None)] * dim
            idx[dim - 1 - ax] = 0 if side == 0 else -1
            bnd[tuple(idx)] = True
    return bnd


def dirichlet_mask(dim: int, cells: tuple, outflow=()) -> np.ndarray:
    """uint8 per unknown: 1 on velocity components of Dirichlet boundary nodes."""
    bnd = _dirichlet_nodes(dim, cells, outflow)
    mask = np.zeros(bnd.shape + (dim + 1,), dtype=np.uint8)
    mask[bnd, :dim] = 1
    return mask.reshape(-1)


@dataclass
class SyntheticSystem:
    problem: Problem
    levels: list              # LevelMatrix per level, coarsest first
    rhs: np.ndarray           # float64 finest-level right-hand side
    dirichlet: np.ndarray     # uint8 finest-level Dirichlet mask

    @property
    def fine(self) -> LevelMatrix:
        return self.levels[-1]

    @property
    def unknowns(self) -> int:
        return int(self.rhs.shape[0])


def build_system(problem: Problem) -> SyntheticSystem:
    """All level matrices, the seeded right-hand side and the Dirichlet mask.

    RHS: numpy default_rng(rhs_seed).uniform(-1, 1, unknowns), zeroed on the
    Dirichlet unknowns.
    """
    conv = ConvectionField(problem.dim, problem.conv_seed) if problem.coef.convection else None
    mats = [assemble_level(problem, c, conv=conv) for c in level_cells(problem)]
    fine = mats[-1]
    mask = dirichlet_mask(problem.dim, fine.cells, problem.outflow)
    rng = np.random.default_rng(problem.rhs_seed)
    rhs = rng.uniform(-1.0, 1.0, size=mask.shape[0])
    rhs[mask.astype(bool)] = 0.0
    return SyntheticSystem(problem=problem, levels=mats, rhs=rhs, dirichlet=mask)


# ----------------------------------------------------------------------------
# ALE extension (problem (3) of Section 4.2): n_c = d
# ----------------------------------------------------------------------------

def ale_fixed_nodes(dim: int, cells: tuple, solid_mask: np.ndarray) -> np.ndarray:
    """Nodes whose deformation is given in the extension problem: the mesh
    boundary (the outer walls do not move) and every node of a solid cell
    (there the deformation is the solid's own, from problem (2)).  Array order
    (z, y, x)."""
    nodes_n = tuple(nk + 1 for nk in cells)
    fixed = _dirichlet_nodes(dim, cells)
    for a in range(2 ** dim):
        pa = tuple((a >> m) & 1 for m in range(dim))
        fixed[_slices(pa, cells)] |= solid_mask
    assert fixed.shape == tuple(reversed(nodes_n))
    return fixed


def assemble_ale_level(problem: Problem, cells: tuple, coarse_cells: Optional[tuple] = None,
                       eliminate: bool = True) -> LevelMatrix:
    """The ALE-extension operator on one level: the harmonic extension of the
    solid deformation into the fluid, one Q1 Laplacian per displacement
    component, (grad u_c, grad phi_c) summed over the fluid cells (2^d-point
    Gauss quadrature).  Rows and columns of the fixed nodes (ale_fixed_nodes)
    are those of the identity; their given values enter through the
    right-hand side.  eliminate=False returns the operator before that step
    (every row and column as assembled), whose free rows carry the coupling
    E_{f,i} of the extension equation to the given values."""
    dim = problem.dim
    nc = dim
    na = 2 ** dim
    h = 1.0 / cells[0]
    nodes_n = tuple(nk + 1 for nk in cells)
    nshape = tuple(reversed(nodes_n))
    nst = 3 ** dim
    solid = solid_cells(problem, cells, coarse_cells)
    fluid = (~solid).astype(np.float64)
    _, w, psi, dpsi = reference_element(dim)
    G = h ** (dim - 2) * np.einsum("q,qam,qbm->ab", w, dpsi, dpsi)
    eye = np.eye(nc)
    S = np.zeros(nshape + (nst, nc, nc))
    for a in range(na):
        pa = tuple((a >> m) & 1 for m in range(dim))
        rows = _slices(pa, cells)
        for b in range(na):
            pb = tuple((b >> m) & 1 for m in range(dim))
            s = sum((pb[m] - pa[m] + 1) * 3 ** m for m in range(dim))
            S[rows + (s,)] += (fluid * G[a, b])[..., None, None] * eye
    if not eliminate:
        return _stencil_to_bsr(S, dim, cells, nc)
    fixed = ale_fixed_nodes(dim, cells, solid)
    S[fixed] = 0.0
    offs = _offsets(dim)
    for s, o in enumerate(offs):
        src, dst = [], []
        for m in reversed(range(dim)):
            lo = max(0, -o[m])
            hi = nodes_n[m] - max(0, o[m])
            dst.append(slice(lo, hi))
            src.append(slice(lo + o[m], hi + o[m]))
        colf = np.zeros(nshape, dtype=bool)
        colf[tuple(dst)] = fixed[tuple(src)]
        S[..., s, :, :][colf] = 0.0
    center = (nst - 1) // 2
    for i in range(nc):
        S[..., center, i, i][fixed] = 1.0
    return _stencil_to_bsr(S, dim, cells, nc)


def ale_mask(problem: Problem, cells: tuple) -> np.ndarray:
    """uint8 per unknown of the extension problem: 1 on every component of a fixed node."""
    fixed = ale_fixed_nodes(problem.dim, cells, solid_cells(problem, cells))
    return np.repeat(fixed.reshape(-1), problem.dim).astype(np.uint8)


def build_ale_system(problem: Problem) -> SyntheticSystem:
    """All level matrices of the ALE-extension problem (n_c = d), its seeded
    right-hand side (numpy default_rng(rhs_seed).uniform(-1, 1), zero on the
    fixed unknowns) and the fixed-unknown mask."""
    mats = [assemble_ale_level(problem, c) for c in level_cells(problem)]
    mask = ale_mask(problem, mats[-1].cells)
    rng = np.random.default_rng(problem.rhs_seed)
    rhs = rng.uniform(-1.0, 1.0, size=mask.shape[0])
    rhs[mask.astype(bool)] = 0.0
    return SyntheticSystem(problem=problem, levels=mats, rhs=rhs, dirichlet=mask)
