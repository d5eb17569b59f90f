"""Pins of the ALE-extension inputs and of the oracle on them (n_c = d).

Problem (3) of Section 4.2 extends the solid deformation harmonically into
the fluid: one Q1 Laplacian per displacement component on the fluid cells,
the deformation given on the solid's nodes and on the outer boundary.  Each
test checks the generator or the oracle against something they do not
compute themselves: textbook element matrices, a manufactured solution,
structure, and dense direct solves.
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from gen import Problem, build_ale_system, reference_element
from gen.q1fsi import ale_fixed_nodes, assemble_ale_level, solid_cells
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy


def _csr(level):
    nc = level.vals.shape[1]
    return sp.bsr_matrix((level.vals, level.col_idx, level.row_ptr), shape=(level.nodes * nc,) * 2).tocsr()


def _problem(dim, n, levels, solid=True):
    return Problem(dim=dim, n=(n,) * dim, levels=levels,
                   solid=((0, +1, 0.6) if dim == 2 else (2, -1, 0.25)) if solid else None)


def test_q1_laplace_element_textbook():
    """The Q1 stiffness of the unit square / cube: 2d diagonal 2/3, edge
    neighbour -1/6, opposite corner -1/3; 3d diagonal 1/3, edge neighbour 0,
    face diagonal -1/12, body diagonal -1/12 (node a at bits (x, y[, z]))."""
    for dim in (2, 3):
        _, w, psi, dpsi = reference_element(dim)
        G = np.einsum("q,qam,qbm->ab", w, dpsi, dpsi)
        na = 2 ** dim
        for a in range(na):
            for b in range(na):
                diff = bin(a ^ b).count("1")
                want = {2: {0: 2 / 3, 1: -1 / 6, 2: -1 / 3}, 3: {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}}[dim][diff]
                assert abs(G[a, b] - want) < 1e-14, (dim, a, b)


@pytest.mark.parametrize("dim", [2, 3])
def test_ale_structure(dim):
    """Symmetric, identity rows and columns at the fixed nodes (boundary and
    every node of a solid cell), block-diagonal in the components, and
    positive definite."""
    n = 8 if dim == 2 else 4
    p = _problem(dim, n, 2)
    lev = assemble_ale_level(p, p.n)
    A = _csr(lev).toarray()
    assert np.abs(A - A.T).max() == 0.0
    fixed = ale_fixed_nodes(dim, p.n, solid_cells(p, p.n)).reshape(-1)
    nc = dim
    fx = np.repeat(fixed, nc)
    assert fx.sum() > 0 and (~fx).sum() > 0
    assert np.array_equal(A[fx][:, fx], np.eye(int(fx.sum())))
    assert np.abs(A[fx][:, ~fx]).max() == 0.0
    # components do not couple
    comp = np.tile(np.arange(nc), A.shape[0] // nc)
    assert np.abs(A[comp[:, None] != comp[None, :]]).max() == 0.0
    np.linalg.cholesky(A)
    # solid cells contribute nothing: a node of only solid cells is a fixed identity row
    assert (np.diag(A)[~fx] > 0).all()


def test_ale_laplacian_manufactured_second_order():
    """No solid, fixed boundary: u_c = c-th multiple of sin(pi x) sin(pi y)
    solves -Lap u = 2 pi^2 u.  The Q1 solution with the load M f_h (the same
    Gauss quadrature for the mass matrix, assembled here) converges at the
    nodes with order 2."""
    errs = []
    sizes = (8, 16, 32)
    for n in sizes:
        p = _problem(2, n, 1, solid=False)
        lev = assemble_ale_level(p, p.n)
        A = _csr(lev)
        h = 1.0 / n
        nn = n + 1
        xs = np.arange(nn) * h
        X, Y = np.meshgrid(xs, xs, indexing="xy")          # (y, x) array order, node = x + nn y
        u = np.sin(np.pi * X) * np.sin(np.pi * Y)
        f = 2 * np.pi ** 2 * u
        # Q1 mass matrix by the same 2x2 Gauss rule
        _, w, psi, _ = reference_element(2)
        Me = h * h * np.einsum("q,qa,qb->ab", w, psi, psi)
        rows, cols, vals = [], [], []
        for cy in range(n):
            for cx in range(n):
                nodes = [cx + (a & 1) + nn * (cy + (a >> 1)) for a in range(4)]
                for a in range(4):
                    for b in range(4):
                        rows.append(nodes[a]); cols.append(nodes[b]); vals.append(Me[a, b])
        M = sp.csr_matrix((vals, (rows, cols)), shape=(nn * nn,) * 2)
        load = M @ f.reshape(-1)
        fixed = ale_fixed_nodes(2, p.n, solid_cells(p, p.n)).reshape(-1)
        b = np.zeros(2 * nn * nn)
        for c in range(2):
            bc = (c + 1) * load
            bc[fixed] = 0.0
            b[c::2] = bc
        x = spl.spsolve(A.tocsc(), b)
        err = max(np.abs(x[c::2] - (c + 1) * u.reshape(-1)).max() / (c + 1) for c in range(2))
        errs.append(err)
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert min(orders) >= 1.8, (errs, orders)


@pytest.mark.parametrize("dim,n,levels", [(2, 16, 3), (2, 32, 4), (3, 8, 2)])
def test_ale_oracle_solve_matches_direct(dim, n, levels):
    """FGMRES with the Vanka V-cycle on the extension problem reaches the
    dense direct solution."""
    s = build_ale_system(_problem(dim, n, levels))
    h = Hierarchy(s.levels, s.dirichlet)
    x, info = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-10)
    xd = np.linalg.solve(_csr(s.fine).toarray(), s.rhs)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert info["iterations"] <= 10


def test_ale_iterations_bounded_under_refinement():
    """Multigrid on the Laplacian: the counts do not grow with the mesh."""
    its = []
    for n, levels in ((32, 3), (64, 4), (128, 5)):
        s = build_ale_system(_problem(2, n, levels))
        h = Hierarchy(s.levels, s.dirichlet)
        _, info = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8)
        its.append(info["iterations"])
    assert max(its) - min(its) <= 1 and max(its) <= 8, its
