"""Pins of the CPU oracle (and of the input generator) to facts outside the oracle.

Each test checks the oracle against something it does not compute itself:
closed forms, brute force on tiny meshes, dense direct solves, exactness
statements of the paper, or the paper's printed iteration-count pattern.
"""

import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from gen import Coefficients, Problem, build_system, config_problem, reference_element
from gen.q1fsi import assemble_level, dirichlet_mask
from oracle.bsr import BlockMatrix
from oracle.fgmres import fgmres
from oracle.mesh import node_coords, patch_dofs, patch_nodes
from oracle.multigrid import Hierarchy
from oracle.transfer import prolongation
from oracle.vanka import overlap_weights, patch_inverses, patch_matrices, vanka_step

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(dim, n, levels, **kw):
    base = dict(dim=dim, n=(n,) * dim, levels=levels,
                solid=(0, +1, 0.6) if dim == 2 else (2, -1, 0.25))
    base.update(kw)
    return Problem(**base)


# ----------------------------------------------------------------------------
# generator: textbook element matrices and manufactured solutions (P6)
# ----------------------------------------------------------------------------

def test_reference_element_closed_forms():
    """Q1 mass and Laplace element matrices on the unit square (textbook values)."""
    _, w, psi, dpsi = reference_element(2)
    M = np.einsum("q,qa,qb->ab", w, psi, psi)
    G = np.einsum("q,qam,qbm->ab", w, dpsi, dpsi)
    # local nodes (0,0), (1,0), (0,1), (1,1)
    M_ref = np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) / 36.0
    G_ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    np.testing.assert_allclose(M, M_ref, atol=1e-15)
    np.testing.assert_allclose(G, G_ref, atol=1e-15)
    # 3d: mass of the unit cube sums to 1, Laplace rows sum to 0, diagonal 1/3
    _, w3, psi3, dpsi3 = reference_element(3)
    M3 = np.einsum("q,qa,qb->ab", w3, psi3, psi3)
    G3 = np.einsum("q,qam,qbm->ab", w3, dpsi3, dpsi3)
    assert abs(M3.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(G3.sum(axis=1), 0.0, atol=1e-14)
    np.testing.assert_allclose(np.diag(G3), 1.0 / 3.0, atol=1e-14)
    np.testing.assert_allclose(np.diag(M3), 8.0 / 216.0, atol=1e-15)


def _load_vector(dim, cells, f, ncomp):
    """int f . psi_a over the mesh with the 2^d Gauss rule (f returns (..., ncomp))."""
    xi, w, psi, _ = reference_element(dim)
    h = 1.0 / cells[0]
    nn = tuple(c + 1 for c in cells)
    F = np.zeros(tuple(reversed(nn)) + (ncomp,))
    origins = np.stack(np.meshgrid(*[np.arange(c) * h for c in reversed(cells)], indexing="ij")[::-1], -1)
    xq = origins[..., None, :] + h * xi
    fq = f(xq)                                            # cells + (nq, ncomp)
    for a in range(2 ** dim):
        pa = [(a >> m) & 1 for m in range(dim)]
        sl = tuple(slice(p, p + c) for p, c in zip(reversed(pa), reversed(cells)))
        F[sl] += h ** dim * np.einsum("q,q,...qc->...c", w, psi[:, a], fq)
    return F.reshape(-1)


def _mms_error(dim, n, solid, v_exact, p_exact, f, coef, conv):
    problem = Problem(dim=dim, n=(n,) * dim, levels=1, solid=solid, coef=coef)
    lev = assemble_level(problem, (n,) * dim, conv=conv)
    A = BlockMatrix(lev.row_ptr, lev.col_idx, lev.vals).csr.tolil()
    nc = dim + 1
    b = _load_vector(dim, (n,) * dim, f, nc)
    mask = dirichlet_mask(dim, (n,) * dim).astype(bool)
    b[mask] = 0.0
    # pin the pressure at node 0 (it is fixed only up to a constant here)
    A[dim, :] = 0.0
    A[dim, dim] = 1.0
    X = node_coords((n,) * dim) / n
    b[dim] = p_exact(X[0:1])[0]
    x = sp.linalg.spsolve(A.tocsr(), b).reshape(-1, nc)
    err = np.abs(x[:, :dim] - v_exact(X)).max()
    return err / np.abs(v_exact(X)).max()


@pytest.mark.parametrize("case", ["fluid", "solid"])
def test_mms_second_order_2d(case):
    """Manufactured solutions converge at second order: the assembled operator is
    the stated PDE (a dropped term, wrong sign or transposed gradient breaks it)."""
    sym = pytest.importorskip("sympy")
    X, Y = sym.symbols("x y")
    coef = Coefficients()
    k, nu = coef.k, coef.nu
    if case == "fluid":
        psi = sym.sin(sym.pi * X) ** 2 * sym.sin(sym.pi * Y) ** 2
        v = [sym.diff(psi, Y), -sym.diff(psi, X)]                      # divergence free
        p = sym.cos(sym.pi * X) * sym.cos(sym.pi * Y)
        bconst = (0.6, -0.8)
        f = [v[i] - k * nu * (sym.diff(v[i], X, 2) + sym.diff(v[i], Y, 2))
             + k * (bconst[0] * sym.diff(v[i], X) + bconst[1] * sym.diff(v[i], Y))
             + k * sym.diff(p, [X, Y][i]) for i in range(2)]
        solid = None
        conv = lambda x: np.broadcast_to(np.array(bconst), x.shape)
    else:
        v = [sym.sin(sym.pi * X) * sym.sin(sym.pi * Y), sym.sin(2 * sym.pi * X) * sym.sin(sym.pi * Y)]
        p = sym.Integer(0)
        div = sym.diff(v[0], X) + sym.diff(v[1], Y)
        kmu, klam = coef.kmu_s, coef.klam_s
        f = [v[i] - k * kmu * (sym.diff(v[i], X, 2) + sym.diff(v[i], Y, 2))
             - k * (kmu + klam) * sym.diff(div, [X, Y][i]) for i in range(2)]
        solid = (0, +1, -1.0)
        conv = None
    fv = [sym.lambdify((X, Y), fi, "numpy") for fi in f]
    vv = [sym.lambdify((X, Y), vi, "numpy") for vi in v]
    pv = sym.lambdify((X, Y), p, "numpy")

    def F(x):
        out = np.zeros(x.shape[:-1] + (3,))
        for i in range(2):
            out[..., i] = fv[i](x[..., 0], x[..., 1])
        return out

    def V(x):
        return np.stack([np.broadcast_to(vv[i](x[..., 0], x[..., 1]), x.shape[:-1]) for i in range(2)], -1)

    def P(x):
        return np.broadcast_to(pv(x[..., 0], x[..., 1]), x.shape[:-1])

    errs = [_mms_error(2, n, solid, V, P, F, coef, conv) for n in (16, 32, 64, 128)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert errs[-1] < 1e-2
    assert orders[-1] > 1.8, (errs, orders)


# ----------------------------------------------------------------------------
# structure invariants (P8)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_structure_invariants(dim):
    n = 8
    problem = small_problem(dim, n, 2)
    sysm = build_system(problem)
    fine = sysm.fine
    nc = dim + 1
    A = BlockMatrix(fine.row_ptr, fine.col_idx, fine.vals).dense()
    mask = sysm.dirichlet.astype(bool)
    # Dirichlet rows and columns are identity
    idx = np.nonzero(mask)[0]
    np.testing.assert_array_equal(A[idx][:, idx], np.eye(idx.size))
    A_off = A.copy()
    A_off[idx, idx] = 0.0
    assert np.all(A_off[idx, :] == 0.0) and np.all(A_off[:, idx] == 0.0)
    # no velocity-pressure coupling at nodes that touch only solid cells
    X = node_coords(fine.cells) / n
    if dim == 2:
        deep_solid = X[:, 0] > 0.5 + 1e-12       # ancestor grid 4x4: solid cells x in [0.5, 1]
    else:
        deep_solid = X[:, 2] < 0.25 - 1e-12      # ancestor grid 4^3: solid cells z in [0, 0.25]
    assert deep_solid.sum() > 0
    rows_p = np.nonzero(deep_solid)[0] * nc + dim
    for r in rows_p:
        vel_cols = [c for c in np.nonzero(A[r])[0] if c % nc != dim]
        assert not vel_cols
    # patch counts and multiplicities: interior vertex in 2^d patches
    pn = patch_nodes(fine.cells)
    assert pn.shape == ((n // 2) ** dim, 3 ** dim)
    mult = np.bincount(pn.reshape(-1), minlength=(n + 1) ** dim)
    coords = node_coords(fine.cells)
    expect = np.ones(coords.shape[0], dtype=int)
    for m in range(dim):
        c = coords[:, m]
        expect *= np.where((c % 2 == 0) & (c > 0) & (c < n), 2, 1)
    np.testing.assert_array_equal(mult, expect)
    # Q1 node-adjacency pattern size
    assert fine.col_idx.size == (3 * (n + 1) - 2) ** dim


# ----------------------------------------------------------------------------
# block matrix product (P5)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_spmv_against_blockwise_loop(dim):
    sysm = build_system(small_problem(dim, 4, 1))
    lev = sysm.fine
    A = BlockMatrix(lev.row_ptr, lev.col_idx, lev.vals)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(A.size)
    nc = lev.ncomp
    y = np.zeros(A.size)
    for i in range(lev.nodes):
        for k in range(lev.row_ptr[i], lev.row_ptr[i + 1]):
            j = lev.col_idx[k]
            for r in range(nc):
                for c in range(nc):
                    y[i * nc + r] += lev.vals[k, r, c] * x[j * nc + c]
    np.testing.assert_allclose(A.matvec(x), y, rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------------------
# transfers (P4)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("coarse", [(3, 2), (2, 2, 3)])
def test_prolongation_reproduces_q1(coarse):
    dim = len(coarse)
    nc = dim + 1
    P = prolongation(coarse, nc)
    fine = tuple(2 * c for c in coarse)
    Xc = node_coords(coarse) / np.array(coarse, dtype=float)
    Xf = node_coords(fine) / np.array(fine, dtype=float)
    rng = np.random.default_rng(3)
    for _ in range(3):
        coef = rng.standard_normal((nc, 2 ** dim))

        def q1(X):
            out = np.zeros((X.shape[0], nc))
            for t in range(2 ** dim):
                mono = np.ones(X.shape[0])
                for m in range(dim):
                    if (t >> m) & 1:
                        mono = mono * X[:, m]
                out += coef[:, t][None, :] * mono[:, None]
            return out.reshape(-1)

        np.testing.assert_allclose(P @ q1(Xc), q1(Xf), rtol=1e-13, atol=1e-13)
    # partition of unity and the 1/2^j weights
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-15)
    vals = np.unique(np.round(P.data, 15))
    assert set(vals.tolist()) <= {1.0, 0.5, 0.25, 0.125}


# ----------------------------------------------------------------------------
# Vanka smoother (P1 and brute force)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_single_patch_vanka_is_exact_solve(dim):
    """One patch covering the mesh: Eq. (vanka) with omega = 1 is the exact solve.

    (A solid half keeps the pressure constant out of the kernel: with velocity
    Dirichlet data on the whole boundary an all-fluid patch is singular.)"""
    sysm = build_system(small_problem(dim, 2, 1, solid=(dim - 1, -1, 0.5)))
    lev = sysm.fine
    A = BlockMatrix(lev.row_ptr, lev.col_idx, lev.vals)
    dofs = patch_dofs(lev.cells, lev.ncomp)
    Ainv = patch_inverses(patch_matrices(A, lev.cells))
    wgt = overlap_weights(dofs, A.size)
    b = sysm.rhs + 0.1
    ref = np.linalg.solve(A.dense(), b)
    x = vanka_step(A, Ainv, dofs, b, np.zeros_like(b), 1.0, wgt)
    np.testing.assert_allclose(x, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())
    x8 = vanka_step(A, Ainv, dofs, b, np.zeros_like(b), 0.8, wgt)
    np.testing.assert_allclose(x8, 0.8 * ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(np.einsum("pij,pjk->pik", Ainv, patch_matrices(A, lev.cells)),
                               np.eye(dofs.shape[1])[None], atol=1e-9)


@pytest.mark.parametrize("dim,n,weighting", [(2, 4, "average"), (2, 6, "sum"), (3, 4, "average")])
def test_vanka_step_against_bruteforce(dim, n, weighting):
    """Eq. (vanka) with patch dof sets found by coordinates and dense solves per patch."""
    sysm = build_system(small_problem(dim, n, 1))
    lev = sysm.fine
    A = BlockMatrix(lev.row_ptr, lev.col_idx, lev.vals)
    Ad = A.dense()
    nc = lev.ncomp
    rng = np.random.default_rng(11)
    b = rng.standard_normal(A.size)
    x0 = rng.standard_normal(A.size)
    coords = node_coords(lev.cells)
    d = b - Ad @ x0
    corr = np.zeros(A.size)
    count = np.zeros(A.size)
    for origin in itertools.product(*[range(0, c, 2) for c in lev.cells]):
        inside = np.all((coords >= np.array(origin)) & (coords <= np.array(origin) + 2), axis=1)
        dof = (np.nonzero(inside)[0][:, None] * nc + np.arange(nc)).reshape(-1)
        corr[dof] += np.linalg.solve(Ad[np.ix_(dof, dof)], d[dof])
        count[dof] += 1
    wgt = 1.0 / count if weighting == "average" else np.ones(A.size)
    ref = x0 + 0.8 * wgt * corr
    dofs = patch_dofs(lev.cells, nc)
    Ainv = patch_inverses(patch_matrices(A, lev.cells))
    got = vanka_step(A, Ainv, dofs, b, x0, 0.8, overlap_weights(dofs, A.size, weighting))
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


# ----------------------------------------------------------------------------
# FGMRES (minimal residual property) and the V-cycle (P3)
# ----------------------------------------------------------------------------

def test_fgmres_is_minimal_residual():
    """With M = I, the j-th FGMRES estimate is min ||b - A y|| over the Krylov space."""
    rng = np.random.default_rng(2)
    n = 12
    A = np.eye(n) * 3 + rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    for j in range(1, 8):
        hist = []
        x, info = fgmres(lambda v: A @ v, lambda v: v, b, rtol=0.0, restart=j, maxit=j, history=hist)
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(j)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        best = np.linalg.norm(b - A @ Q @ y) / np.linalg.norm(b)
        assert abs(hist[-1] - best) < 1e-10
        assert abs(np.linalg.norm(b - A @ x) / np.linalg.norm(b) - best) < 1e-10
    x, info = fgmres(lambda v: A @ v, lambda v: v, b, rtol=1e-12, restart=n)
    assert info["converged"] and info["iterations"] <= n


def test_single_level_fgmres_converges_in_one_step():
    sysm = build_system(small_problem(2, 8, 1))
    h = Hierarchy(sysm.levels, sysm.dirichlet)
    x, info = fgmres(h.fine.A.matvec, h.vcycle, sysm.rhs, rtol=1e-8)
    assert info["iterations"] == 1 and info["converged"]


@pytest.mark.parametrize("dim", [2, 3])
def test_two_level_coarse_correction_bruteforce(dim):
    """nu1 = nu2 = 0: the V-cycle is P A_c^{-1} P^T with the Dirichlet entries zeroed;
    P is built here by coordinates, independently of the oracle's Kronecker form."""
    n = 4
    sysm = build_system(small_problem(dim, n, 2, solid=(dim - 1, -1, 0.5)))
    h = Hierarchy(sysm.levels, sysm.dirichlet, nu1=0, nu2=0)
    nc = dim + 1
    fcells = sysm.levels[1].cells
    ccells = sysm.levels[0].cells
    Xf = node_coords(fcells)
    Xc = node_coords(ccells)
    P = np.zeros((Xf.shape[0] * nc, Xc.shape[0] * nc))
    for i, xf in enumerate(Xf):
        for j, xc in enumerate(Xc):
            w = 1.0
            for m in range(dim):
                dist = abs(xf[m] - 2 * xc[m])
                w *= 1.0 if dist == 0 else (0.5 if dist == 1 else 0.0)
            if w:
                for c in range(nc):
                    P[i * nc + c, j * nc + c] = w
    fmask = sysm.dirichlet.astype(bool)
    cmask = fmask.reshape(-1, nc)[[int(np.argmin(np.abs(Xf - 2 * xc).sum(1))) for xc in Xc]].reshape(-1)
    Ac = BlockMatrix(sysm.levels[0].row_ptr, sysm.levels[0].col_idx, sysm.levels[0].vals).dense()
    rng = np.random.default_rng(4)
    r = rng.standard_normal(Xf.shape[0] * nc)
    rc = P.T @ r
    rc[cmask] = 0.0
    ref = P @ np.linalg.solve(Ac, rc)
    ref[fmask] = 0.0
    np.testing.assert_allclose(h.vcycle(r), ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_vcycle_is_linear_and_stateless(dim):
    """A V-cycle that starts every level from zero (Sec. 4.3 (II)) applies one
    fixed linear operator to its input: V(a r1 + b r2) = a V(r1) + b V(r2) to
    rounding, and a repeated call returns the same vector bit for bit (no state
    carried between applications).  A lost zero start or an iterate kept from
    the previous call breaks either; many right-hand sides can therefore be
    preconditioned column by column."""
    sysm = build_system(small_problem(dim, 8 if dim == 2 else 4, 2))
    h = Hierarchy(sysm.levels, sysm.dirichlet)
    rng = np.random.default_rng(9)
    mask = sysm.dirichlet.astype(bool)
    r1, r2 = rng.standard_normal(sysm.rhs.size), rng.standard_normal(sysm.rhs.size)
    r1[mask] = 0.0
    r2[mask] = 0.0
    a, b = 1.7, -0.3
    z1 = h.vcycle(r1)
    z2 = h.vcycle(r2)
    lhs = h.vcycle(a * r1 + b * r2)
    assert np.linalg.norm(lhs - (a * z1 + b * z2)) <= 1e-12 * np.linalg.norm(a * z1 + b * z2)
    assert np.array_equal(h.vcycle(r1), z1)
    assert np.linalg.norm(z1) > 0


def _dense_patch_smoother(Ad, cells, nc, omega, weighting):
    """S = omega W sum_i R_i^T (R_i A R_i^T)^{-1} R_i as a dense matrix, the patch
    dof sets found from node coordinates (the 3^d nodes of each 2^d-cell block)."""
    coords = node_coords(cells)
    n = Ad.shape[0]
    S = np.zeros((n, n))
    count = np.zeros(n)
    for origin in itertools.product(*[range(0, c, 2) for c in cells]):
        inside = np.all((coords >= np.array(origin)) & (coords <= np.array(origin) + 2), axis=1)
        dof = (np.nonzero(inside)[0][:, None] * nc + np.arange(nc)).reshape(-1)
        S[np.ix_(dof, dof)] += np.linalg.inv(Ad[np.ix_(dof, dof)])
        count[dof] += 1
    w = 1.0 / count if weighting == "average" else np.ones(n)
    return omega * w[:, None] * S


def _dense_interpolation(fcells, ccells, nc):
    """Q1 nodal interpolation by coordinates: fine node x gets weight
    prod_m (1 if x_m = 2 X_m, 1/2 if |x_m - 2 X_m| = 1) from coarse node X."""
    Xf, Xc = node_coords(fcells), node_coords(ccells)
    dist = np.abs(Xf[:, None, :] - 2 * Xc[None, :, :])
    w = np.prod(np.where(dist == 0, 1.0, np.where(dist == 1, 0.5, 0.0)), axis=2)
    return np.kron(w, np.eye(nc))


def _dense_vcycle_matrix(sysm, nu1, nu2, omega, weighting):
    """The V(nu1, nu2) preconditioner as one dense matrix, through the error
    propagation identity of a consistent linear iteration started from zero:
    z = M b with M = (I - E) A^{-1}, E = (I - S A)^nu2 (I - C A) (I - S A)^nu1,
    C = Z_f P M_c Z_c P^T (the coarse-grid correction with the Dirichlet
    entries of the restricted residual and of the prolonged correction
    zeroed), M_0 = A_0^{-1}.  Nothing here steps through the cycle."""
    nc = sysm.problem.ncomp
    lv = sysm.levels
    mats = [BlockMatrix(l.row_ptr, l.col_idx, l.vals).dense() for l in lv]
    # Dirichlet unknowns of every level: coarse node X is fine node 2X
    masks = [None] * len(lv)
    masks[-1] = sysm.dirichlet.astype(bool)
    for lev in range(len(lv) - 1, 0, -1):
        Xf, Xc = node_coords(lv[lev].cells), node_coords(lv[lev - 1].cells)
        fine_of = [int(np.argmin(np.abs(Xf - 2 * xc).sum(1))) for xc in Xc]
        masks[lev - 1] = masks[lev].reshape(-1, nc)[fine_of].reshape(-1)
    M = np.linalg.inv(mats[0])
    for lev in range(1, len(lv)):
        A = mats[lev]
        n = A.shape[0]
        I = np.eye(n)
        S = _dense_patch_smoother(A, lv[lev].cells, nc, omega, weighting)
        P = _dense_interpolation(lv[lev].cells, lv[lev - 1].cells, nc)
        Zf = np.diag((~masks[lev]).astype(float))
        Zc = np.diag((~masks[lev - 1]).astype(float))
        C = Zf @ P @ M @ Zc @ P.T
        Es = I - S @ A
        E = np.linalg.matrix_power(Es, nu2) @ (I - C @ A) @ np.linalg.matrix_power(Es, nu1)
        M = (I - E) @ np.linalg.inv(A)
    return M


@pytest.mark.parametrize("dim,n,levels", [(2, 8, 2), (2, 16, 3), (3, 4, 2), (3, 8, 3)])
@pytest.mark.parametrize("nu,omega,weighting", [((1, 1), 0.8, "average"), ((2, 2), 0.8, "average"),
                                                ((2, 1), 0.8, "average"), ((1, 2), 0.3, "sum")])
def test_vcycle_composition_against_error_propagation(dim, n, levels, nu, omega, weighting):
    """The oracle's V(nu1, nu2) cycle (Sec. 4.3 (II) with the smoother of
    Eq. (vanka)) on 2 and 3 levels equals the dense operator (I - E) A^{-1}
    built from the error propagation matrix of its stages.  The dense side
    finds patch dofs, interpolation weights and coarse Dirichlet entries from
    node coordinates.  Restricting b instead of b - A x, post-smoothing the
    uncorrected iterate, swapping nu1 and nu2, or dropping a Dirichlet zeroing
    each change M."""
    sysm = build_system(small_problem(dim, n, levels, solid=(dim - 1, -1, 0.5)))
    h = Hierarchy(sysm.levels, sysm.dirichlet, nu1=nu[0], nu2=nu[1], omega=omega, weighting=weighting)
    M = _dense_vcycle_matrix(sysm, nu[0], nu[1], omega, weighting)
    rng = np.random.default_rng(21)
    for _ in range(2):
        r = rng.standard_normal(sysm.rhs.size)
        ref = M @ r
        got = h.vcycle(r)
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("slip", ["restrict_b", "post_from_uncorrected", "swap_nu"])
def test_vcycle_composition_pin_detects_slips(slip, monkeypatch):
    """Each plausible slip, planted in the oracle's V-cycle on the CPU, moves
    it away from the error-propagation operator by far more than the pin's
    tolerance (the pin above is not vacuous).  Dropping the Dirichlet zeroing
    of the prolonged correction is not among them: with velocity Dirichlet
    data on the whole boundary the coarse correction already vanishes on the
    boundary nodes (identity rows, zeroed residual entries, and fine boundary
    nodes interpolated from coarse boundary nodes only), so that zeroing does
    not change the result on these meshes."""
    sysm = build_system(small_problem(2, 8, 2, solid=(1, -1, 0.5)))
    M = _dense_vcycle_matrix(sysm, 2, 1, 0.8, "average")
    h = Hierarchy(sysm.levels, sysm.dirichlet, nu1=2, nu2=1)
    if slip == "restrict_b":
        def restrict_residual(lev, b, x):
            rc = h.levels[lev].P.T @ b
            rc[h.levels[lev - 1].mask] = 0.0
            return rc
        monkeypatch.setattr(h, "restrict_residual", restrict_residual)
    elif slip == "post_from_uncorrected":
        orig = h.prolongate
        monkeypatch.setattr(h, "prolongate", lambda lev, ec: 0.0 * orig(lev, ec))
    else:
        h.nu1, h.nu2 = 1, 2
    r = np.random.default_rng(21).standard_normal(sysm.rhs.size)
    ref = M @ r
    assert np.linalg.norm(h.vcycle(r) - ref) > 1e-8 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------
# whole solve against dense direct solves (P2)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n,levels", [(2, 4, 1), (2, 8, 2), (2, 16, 3), (3, 4, 1), (3, 8, 2)])
def test_solve_matches_dense_direct(dim, n, levels):
    sysm = build_system(small_problem(dim, n, levels))
    h = Hierarchy(sysm.levels, sysm.dirichlet)
    A = h.fine.A.dense()
    b = sysm.rhs
    rtol = 1e-10       # a direct LU solve of these (kappa ~ 1e8-1e9) systems attains ~3e-12
    x, info = fgmres(h.fine.A.matvec, h.vcycle, b, rtol=rtol)
    assert info["converged"]
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= rtol * 1.01
    ref = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= cond * rtol


# ----------------------------------------------------------------------------
# grid-independent multigrid (P7), against the paper's printed pattern
# ----------------------------------------------------------------------------

def _paper_max_increase():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_gmres_per_newton.txt"))
            if l.strip() and not l.startswith("#")]
    inc = 0.0
    for dim in ("2", "3"):
        vals = [float(r[2]) for r in rows if r[0] == dim]
        inc = max(inc, max(b - a for a, b in zip(vals, vals[1:])))
    return inc


@pytest.mark.parametrize("dim,sizes", [(2, (16, 32, 64, 128)), (3, (8, 16))])
def test_iteration_counts_bounded_under_refinement(dim, sizes):
    bound = _paper_max_increase()
    assert abs(bound - 4.54) < 1e-9
    counts = []
    for n in sizes:
        levels = int(math.log2(n)) - 1
        sysm = build_system(small_problem(dim, n, levels))
        h = Hierarchy(sysm.levels, sysm.dirichlet)
        _, info = fgmres(h.fine.A.matvec, h.vcycle, sysm.rhs, rtol=1e-8)
        assert info["converged"]
        counts.append(info["iterations"])
    incs = [b - a for a, b in zip(counts, counts[1:])]
    assert max(incs) <= math.ceil(bound), counts
    assert max(counts) <= 30, counts
