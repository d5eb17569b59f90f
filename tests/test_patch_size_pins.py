"""Pins of the oracle's Vanka smoother with patches of two sizes (Section
5.5.1, Table "testVankaBlock": small patches of one element's unknowns, large
patches of four (2d) or eight (3d) adjacent elements; here 2^d and 4^d Q1
cells, 27 / 75 unknowns in 2d and 108 / 500 in 3d)."""

import itertools

import numpy as np
import pytest

from gen import Problem, build_system
from gen.q1fsi import solid_cells
from oracle.bsr import BlockMatrix
from oracle.fgmres import fgmres
from oracle.mesh import block_nodes, coarse_cell_mask, node_coords, patch_blocks
from oracle.multigrid import Hierarchy
from oracle.vanka import group_weights, patch_groups, vanka_step_groups


def _problem(dim, n, levels, solid=None):
    return Problem(dim=dim, n=(n,) * dim, levels=levels,
                   solid=solid or ((0, +1, 0.5) if dim == 2 else (2, -1, 0.5)))


@pytest.mark.parametrize("cells", [(8, 8), (12, 8), (8, 8, 8), (8, 4, 12)])
def test_patches_partition_the_cells(cells):
    """Every cell lies in exactly one patch; large patches sit exactly on the
    4-aligned blocks whose cells are all flagged."""
    rng = np.random.default_rng(3)
    shape = tuple(reversed(cells))
    mask = rng.random(shape) < 0.6
    mask[(slice(0, 4),) * len(cells)] = True          # at least one full block
    blocks = patch_blocks(cells, mask)
    cover = np.zeros(shape, dtype=int)
    for org, size in blocks:
        sl = tuple(slice(o, o + size) for o in reversed(org))
        cover[sl] += 1
        if size == 4:
            assert all(o % 4 == 0 for o in org) and mask[sl].all()
        else:
            assert all(o % 2 == 0 for o in org)
    assert (cover == 1).all()
    full = 0
    for o in itertools.product(*[range(0, c - 3, 4) for c in reversed(cells)]):
        full += mask[tuple(slice(v, v + 4) for v in o)].all()
    assert sum(s == 4 for _, s in blocks) == full >= 1
    # the patch of a block holds its (size + 1)^d nodes
    org, size = [b for b in blocks if b[1] == 4][0]
    X = node_coords(cells)[block_nodes(cells, org, size)]
    assert X.shape[0] == 5 ** len(cells) and (X.min(0) == np.array(org)).all() and (X.max(0) == np.array(org) + 4).all()


def test_coarse_cell_mask():
    m = np.zeros((8, 8), dtype=bool)
    m[:, 4:] = True
    m[0, 4] = False
    c = coarse_cell_mask(m)
    assert c.shape == (4, 4) and c[:, 2:].sum() == 7 and not c[0, 2] and not c[:, :2].any()


@pytest.mark.parametrize("dim", [2, 3])
def test_single_large_patch_is_the_exact_solve(dim):
    """One large patch covering a 4^d-cell mesh: Eq. (vanka) with omega = 1 is
    the exact solve (75 unknowns in 2d, 500 in 3d)."""
    s = build_system(_problem(dim, 4, 1))
    lev = s.fine
    A = BlockMatrix(lev.row_ptr, lev.col_idx, lev.vals)
    groups = patch_groups(A, lev.cells, np.ones(tuple(reversed(lev.cells)), dtype=bool))
    assert len(groups) == 1 and groups[0][0].shape == (1, 5 ** dim * (dim + 1))
    b = s.rhs + 0.1
    w = group_weights(groups, A.size)
    x = vanka_step_groups(A, groups, b, np.zeros_like(b), 1.0, w)
    ref = np.linalg.solve(A.dense(), b)
    np.testing.assert_allclose(x, ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("dim,n,weighting", [(2, 8, "average"), (2, 12, "sum"), (3, 8, "average")])
def test_mixed_vanka_step_against_bruteforce(dim, n, weighting):
    """Eq. (vanka) with both patch sizes: patch dof sets found from node
    coordinates, a dense solve per patch, corrections summed per unknown."""
    p = _problem(dim, n, 1)
    s = build_system(p)
    lev = s.fine
    A = BlockMatrix(lev.row_ptr, lev.col_idx, lev.vals)
    Ad = A.dense()
    nc = lev.ncomp
    mask = solid_cells(p, lev.cells)
    assert mask.any() and not mask.all()
    rng = np.random.default_rng(11)
    b, x0 = rng.standard_normal(A.size), rng.standard_normal(A.size)
    coords = node_coords(lev.cells)
    d = b - Ad @ x0
    corr, count = np.zeros(A.size), np.zeros(A.size)
    nlarge = 0
    for origin in itertools.product(*[range(0, c, 2) for c in lev.cells]):
        big = tuple((v // 4) * 4 for v in origin)
        in_big = all(bb + 4 <= c for bb, c in zip(big, lev.cells)) and \
            mask[tuple(slice(v, v + 4) for v in reversed(big))].all()
        if in_big and origin != big:
            continue                               # covered by the large patch at big
        size = 4 if in_big else 2
        nlarge += size == 4
        inside = np.all((coords >= np.array(origin)) & (coords <= np.array(origin) + size), axis=1)
        dof = (np.nonzero(inside)[0][:, None] * nc + np.arange(nc)).reshape(-1)
        corr[dof] += np.linalg.solve(Ad[np.ix_(dof, dof)], d[dof])
        count[dof] += 1
    assert nlarge > 0
    w = 1.0 / count if weighting == "average" else np.ones(A.size)
    ref = x0 + 0.8 * w * corr
    groups = patch_groups(A, lev.cells, mask)
    assert groups[1][0].shape[0] == nlarge
    got = vanka_step_groups(A, groups, b, x0, 0.8, group_weights(groups, A.size, weighting))
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def _mixed_dense_vcycle(s, large, nu1, nu2, omega):
    """The V-cycle with mixed patches as one dense matrix through the error
    propagation identity (as for uniform patches in test_oracle_pins), the
    patches found from coordinates and the large-patch region coarsened by
    'all children flagged'."""
    from test_oracle_pins import _dense_interpolation
    nc = s.problem.ncomp
    lv = s.levels
    masks = [None] * len(lv)
    masks[-1] = s.dirichlet.astype(bool)
    regions = [None] * len(lv)
    regions[-1] = large
    for lev in range(len(lv) - 1, 0, -1):
        Xf, Xc = node_coords(lv[lev].cells), node_coords(lv[lev - 1].cells)
        fine_of = [int(np.argmin(np.abs(Xf - 2 * xc).sum(1))) for xc in Xc]
        masks[lev - 1] = masks[lev].reshape(-1, nc)[fine_of].reshape(-1)
        r = regions[lev]
        c = np.ones(tuple(v // 2 for v in r.shape), dtype=bool)
        for off in itertools.product((0, 1), repeat=r.ndim):
            c &= r[tuple(slice(o, None, 2) for o in off)]
        regions[lev - 1] = c
    mats = [BlockMatrix(l.row_ptr, l.col_idx, l.vals).dense() for l in lv]
    M = np.linalg.inv(mats[0])
    for lev in range(1, len(lv)):
        A = mats[lev]
        n = A.shape[0]
        cells = lv[lev].cells
        coords = node_coords(cells)
        S = np.zeros((n, n))
        count = np.zeros(n)
        reg = regions[lev]
        for origin in itertools.product(*[range(0, c, 2) for c in cells]):
            big = tuple((v // 4) * 4 for v in origin)
            in_big = all(bb + 4 <= c for bb, c in zip(big, cells)) and \
                reg[tuple(slice(v, v + 4) for v in reversed(big))].all()
            if in_big and origin != big:
                continue
            size = 4 if in_big else 2
            inside = np.all((coords >= np.array(origin)) & (coords <= np.array(origin) + size), axis=1)
            dof = (np.nonzero(inside)[0][:, None] * nc + np.arange(nc)).reshape(-1)
            S[np.ix_(dof, dof)] += np.linalg.inv(A[np.ix_(dof, dof)])
            count[dof] += 1
        S = omega * (1.0 / count)[:, None] * S
        P = _dense_interpolation(cells, lv[lev - 1].cells, nc)
        Zf = np.diag((~masks[lev]).astype(float))
        Zc = np.diag((~masks[lev - 1]).astype(float))
        C = Zf @ P @ M @ Zc @ P.T
        Es = np.eye(n) - S @ A
        E = np.linalg.matrix_power(Es, nu2) @ (np.eye(n) - C @ A) @ np.linalg.matrix_power(Es, nu1)
        M = (np.eye(n) - E) @ np.linalg.inv(A)
    return M


@pytest.mark.parametrize("dim,n,levels", [(2, 16, 3), (3, 8, 2)])
def test_mixed_vcycle_against_error_propagation(dim, n, levels):
    p = _problem(dim, n, levels)
    s = build_system(p)
    large = solid_cells(p, p.n)
    h = Hierarchy(s.levels, s.dirichlet, nu1=2, nu2=1, large_cells=large)
    assert any(L.groups is not None for L in h.levels)
    M = _mixed_dense_vcycle(s, large, 2, 1, 0.8)
    r = np.random.default_rng(2).standard_normal(s.rhs.size)
    ref = M @ r
    assert np.linalg.norm(h.vcycle(r) - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("dim,n,levels", [(2, 16, 3), (3, 8, 2)])
def test_mixed_solve_matches_dense_direct(dim, n, levels):
    p = _problem(dim, n, levels)
    s = build_system(p)
    h = Hierarchy(s.levels, s.dirichlet, large_cells=solid_cells(p, p.n))
    A = h.fine.A.dense()
    x, info = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-10)
    assert info["converged"]
    ref = np.linalg.solve(A, s.rhs)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= np.linalg.cond(A) * 1e-10


@pytest.mark.parametrize("dim,n,levels", [(2, 64, 4), (3, 16, 3)])
def test_large_patches_take_fewer_iterations(dim, n, levels):
    """The trend of the paper's patch-size table: large patches everywhere
    need fewer FGMRES iterations than small patches everywhere (there
    12.60 against 20.58 GMRES steps per Newton step)."""
    p = _problem(dim, n, levels, solid=(0, +1, 0.6) if dim == 2 else (2, -1, 0.25))
    s = build_system(p)
    its = {}
    for name, large in (("small", None), ("large", np.ones(tuple(reversed(p.n)), dtype=bool))):
        h = Hierarchy(s.levels, s.dirichlet, large_cells=large)
        _, info = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8)
        assert info["converged"]
        its[name] = info["iterations"]
    assert its["large"] < its["small"], its
