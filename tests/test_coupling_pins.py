"""Pins of the oracle's problems (2) and (3) around the momentum solve.

The three sub-steps of Section 4.2 (momentum, deformation update, extension)
are forward substitution through one block lower-triangular system.  Here
that system is assembled densely and independently (the deformation rows with
the consistent Q1 mass matrix of the solid cells on both sides, the extension
rows with every coupling of the assembled operator, solid cells found from
the coarsest-level centroids) and solved directly; the oracle's sub-steps must reproduce its
solution, with dense and with iterative (FGMRES + V-cycle) inner solves.
A wrong sign or scale of k theta, a missing lifting of the interface values,
a mixed-up component or a wrong node set fails it.
"""

import itertools

import numpy as np
import pytest

from gen import Problem, build_ale_system, build_system, reference_element
from gen.q1fsi import ale_fixed_nodes, assemble_ale_level, solid_cells
from oracle.bsr import BlockMatrix
from oracle.coupling import deformation_update, extension_rhs, linear_newton_step
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy

K_THETA = 0.01


def _problem(dim, n, levels):
    # 3d: solid below z = 0.5, so that a 2-level 4^3 mesh has solid cells
    return Problem(dim=dim, n=(n,) * dim, levels=levels, solid=(0, +1, 0.6) if dim == 2 else (2, -1, 0.5))


def _dense(level):
    return BlockMatrix(level.row_ptr, level.col_idx, level.vals).dense()


def _geometry(p):
    """Solid cells (a cell is solid when the centroid of its ancestor on the
    coarsest level lies in the solid region, so every level resolves the same
    interface), their nodes, the outer-boundary nodes and the consistent Q1
    mass matrix of the solid cells (nodes x nodes)."""
    dim, n = p.dim, p.n[0]
    axis, sign, thr = p.solid
    nn = n + 1
    h = 1.0 / n
    ratio = 2 ** (p.levels - 1)     # fine cells per coarsest cell along an axis
    nodes = nn ** dim
    _, w, psi, _ = reference_element(dim)
    Me = h ** dim * np.einsum("q,qa,qb->ab", w, psi, psi)
    M = np.zeros((nodes, nodes))
    solid_nodes = np.zeros(nodes, dtype=bool)
    for cell in itertools.product(range(n), repeat=dim):     # cell[m] = index along axis m
        centroid = (cell[axis] // ratio + 0.5) * ratio * h
        if sign * (centroid - thr) <= 0:
            continue
        ids = []
        for a in range(2 ** dim):
            idx, stride = 0, 1
            for m in range(dim):
                idx += (cell[m] + ((a >> m) & 1)) * stride
                stride *= nn
            ids.append(idx)
        solid_nodes[ids] = True
        M[np.ix_(ids, ids)] += Me
    boundary = np.zeros(nodes, dtype=bool)
    for idx, coord in enumerate(itertools.product(range(nn), repeat=dim)):
        # itertools varies the last entry fastest; node numbering is x fastest
        c = coord[::-1]
        boundary[idx] = any(v in (0, n) for v in c)
    return solid_nodes, boundary, M


def _monolithic(p, s1, E_full, M, solid_nodes, boundary, b1, r, b5):
    dim = p.dim
    nodes = solid_nodes.size
    N1, N3 = nodes * (dim + 1), nodes * dim
    A1 = _dense(s1.fine)
    Ef = E_full.dense()
    T = np.zeros((N1 + N3, N1 + N3))
    rhs = np.zeros(N1 + N3)
    T[:N1, :N1] = A1
    rhs[:N1] = b1
    cols_s = np.flatnonzero(solid_nodes)
    for node in range(nodes):
        for c in range(dim):
            row = N1 + node * dim + c
            if boundary[node]:
                T[row, N1 + node * dim + c] = 1.0
            elif solid_nodes[node]:
                for m in cols_s:
                    T[row, N1 + m * dim + c] += M[node, m]
                    T[row, m * (dim + 1) + c] -= K_THETA * M[node, m]
                    rhs[row] += M[node, m] * r[m * dim + c]
            else:
                T[row, N1:] = Ef[node * dim + c]
                rhs[row] = b5[node * dim + c]
    y = np.linalg.solve(T, rhs)
    return y[:N1], y[N1:]


@pytest.mark.parametrize("dim,n,levels", [(2, 8, 2), (3, 4, 2)])
def test_sub_steps_equal_the_monolithic_solve(dim, n, levels):
    p = _problem(dim, n, levels)
    s1 = build_system(p)
    s3 = build_ale_system(p)
    E_full = BlockMatrix(*(lambda L: (L.row_ptr, L.col_idx, L.vals))(assemble_ale_level(p, p.n, eliminate=False)))
    solid_nodes, boundary, M = _geometry(p)
    # the centroid-based node sets agree with the generator's fixed set
    fixed = ale_fixed_nodes(dim, p.n, solid_cells(p, p.n)).reshape(-1)
    assert np.array_equal(fixed, solid_nodes | boundary)
    assert (solid_nodes & ~boundary).any() and (~fixed).any()
    rng = np.random.default_rng(21)
    nodes = solid_nodes.size
    r = rng.uniform(-1, 1, nodes * dim)
    r.reshape(nodes, dim)[~(solid_nodes & ~boundary)] = 0.0
    b5 = rng.uniform(-1, 1, nodes * dim)
    b1 = s1.rhs
    w_ref, u_ref = _monolithic(p, s1, E_full, M, solid_nodes, boundary, b1, r, b5)

    A1 = _dense(s1.fine)
    E = _dense(s3.fine)
    w, u = linear_newton_step(lambda b: np.linalg.solve(A1, b), b1, r, K_THETA, solid_nodes & ~boundary,
                              lambda b: np.linalg.solve(E, b), E_full, b5, fixed, dim)
    assert np.linalg.norm(w - w_ref) <= 1e-10 * np.linalg.norm(w_ref)
    assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)

    # the same with the oracle's iterative solves of problems (1) and (3)
    h1 = Hierarchy(s1.levels, s1.dirichlet)
    h3 = Hierarchy(s3.levels, s3.dirichlet)
    w_i, u_i = linear_newton_step(lambda b: fgmres(h1.fine.A.matvec, h1.vcycle, b, rtol=1e-12)[0], b1, r, K_THETA,
                                  solid_nodes & ~boundary,
                                  lambda b: fgmres(h3.fine.A.matvec, h3.vcycle, b, rtol=1e-12)[0], E_full, b5,
                                  fixed, dim)
    assert np.linalg.norm(w_i - w_ref) <= 1e-8 * np.linalg.norm(w_ref)
    assert np.linalg.norm(u_i - u_ref) <= 1e-8 * np.linalg.norm(u_ref)


def test_deformation_update_is_the_mass_matrix_solve():
    """Both sides of problem (2) carry the mass matrix of the solid cells:
    solving M du = M r + k theta M dv on the solid and interface nodes gives the
    vector addition, componentwise on the velocity components only."""
    p = _problem(2, 8, 1)
    solid_nodes, boundary, M = _geometry(p)
    S = solid_nodes & ~boundary
    rng = np.random.default_rng(5)
    nodes = S.size
    r = rng.uniform(-1, 1, nodes * 2)
    dv = rng.uniform(-1, 1, nodes * 3)
    du = deformation_update(r, dv, K_THETA, S, 2)
    idx = np.flatnonzero(S)
    Mss = M[np.ix_(idx, idx)]
    for c in range(2):
        rhs = Mss @ (r.reshape(nodes, 2)[idx, c] + K_THETA * dv.reshape(nodes, 3)[idx, c])
        np.testing.assert_allclose(du.reshape(nodes, 2)[idx, c], np.linalg.solve(Mss, rhs), rtol=1e-12, atol=1e-14)
    assert np.count_nonzero(du.reshape(nodes, 2)[~S]) == 0


def test_extension_rhs_lifts_the_fixed_values():
    """With g on the fixed nodes, the reduced system's solution equals the
    solution of the unreduced operator's free rows with those values fixed."""
    p = _problem(2, 8, 2)
    s3 = build_ale_system(p)
    E_full = BlockMatrix(*(lambda L: (L.row_ptr, L.col_idx, L.vals))(assemble_ale_level(p, p.n, eliminate=False)))
    fixed = ale_fixed_nodes(2, p.n, solid_cells(p, p.n)).reshape(-1)
    rng = np.random.default_rng(6)
    nu = fixed.size * 2
    g = rng.uniform(-1, 1, nu)
    b5 = rng.uniform(-1, 1, nu)
    u = np.linalg.solve(_dense(s3.fine), extension_rhs(E_full, b5, fixed, g, 2))
    F = np.repeat(fixed, 2)
    assert np.array_equal(u[F], g[F])
    Ef = E_full.dense()
    res = Ef[~F] @ u - b5[~F]
    assert np.abs(res).max() <= 1e-10 * (np.abs(Ef).max() * np.abs(u).max() + np.abs(b5).max())
