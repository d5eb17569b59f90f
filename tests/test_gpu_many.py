"""Multi-vector V-cycles and solves on the GPU (many right-hand sides against
one factored hierarchy).

nmg_vcycle_many and nmg_solve_many compute every column with the kernels'
per-column arithmetic of the single-vector path, so each column must equal
nmg_vcycle / nmg_solve on that column alone bit for bit.  Single-column
results are themselves checked against the oracle here (V-cycle within the
FP32 / BF16 tolerances of the single-vector tests, solves to the method's
residual tolerance), so the chain reaches the oracle without trusting the
multi-vector path.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import Problem, build_ale_system, build_system
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy

pytestmark = pytest.mark.gpu

CASES = {
    "2d_32x32_3lev": (Problem(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6)), False),
    "2d_24x40_3lev": (Problem(dim=2, n=(24, 40), levels=3, solid=(0, +1, 0.6)), False),
    "3d_8x12x16_3lev": (Problem(dim=3, n=(8, 12, 16), levels=3, solid=(2, -1, 0.5)), False),
    "ale_2d_32x32_3lev": (Problem(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6)), True),
    "ale_3d_8x12x16_3lev": (Problem(dim=3, n=(8, 12, 16), levels=3, solid=(2, -1, 0.5)), True),
}


@pytest.fixture(scope="module")
def nmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300 import nmg as lib
    return lib


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, (p, ale) in CASES.items():
        s = build_ale_system(p) if ale else build_system(p)
        out[name] = (s, Hierarchy(s.levels, s.dirichlet), ale)
    return out


@pytest.fixture(scope="module")
def sessions(nmg, built):
    from paper_1904_02401_gb300.session import Session
    out = {}
    for name, (s, _, ale) in built.items():
        out[name] = Session(s.problem.dim, s.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels],
                            s.dirichlet, ncomp=s.problem.dim if ale else None)
    yield out
    for v in out.values():
        v.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _columns(s, nrhs, seed):
    """nrhs right-hand sides: the workload's own, then seeded random vectors
    of the same size (Dirichlet entries zero), with different scales."""
    rng = np.random.default_rng(seed)
    mask = np.asarray(s.dirichlet, dtype=bool).reshape(-1)
    cols = [s.rhs]
    for k in range(1, nrhs):
        v = rng.uniform(-1.0, 1.0, s.rhs.size) * (10.0 ** (k % 3 - 1))
        v[mask] = 0.0
        cols.append(v)
    return np.stack(cols)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("nrhs", [1, 3, 4, 5, 8, 11])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_vcycle_many_equals_single(nmg, built, sessions, case, prec, nrhs, use_graph):
    from paper_1904_02401_gb300.session import solve_opts
    s, h, _ = built[case]
    S = sessions[case]
    R = torch.from_numpy(_columns(s, nrhs, 11).astype(np.float32)).cuda()
    Z = torch.full_like(R, float("nan"))
    nmg.check(nmg.nmg_vcycle_many(S.handle, solve_opts(precision=prec, use_graph=use_graph), nrhs, R, Z))
    for k in range(nrhs):
        z = torch.zeros_like(R[k])
        nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=0, engine=nmg.NMG_ENGINE_KERNELS),
                                 R[k].contiguous(), z))
        assert torch.equal(Z[k], z), (case, k)
    # and the first column against the oracle's FP64 V-cycle
    r = R[0].cpu().numpy().astype(np.float64)
    tol = 1e-3 if prec == 1 else 5e-2
    assert rel(Z[0].cpu().numpy().astype(np.float64), h.vcycle(r)) < tol


@pytest.mark.parametrize("case", ["2d_32x32_3lev", "3d_8x12x16_3lev"])
def test_vcycle_many_engines_agree(nmg, built, sessions, case):
    """The single-vector engines agree bitwise with one another, so a column of
    the multi-vector V-cycle equals the autotuned single V-cycle too."""
    from paper_1904_02401_gb300.session import solve_opts
    s, _, _ = built[case]
    S = sessions[case]
    R = torch.from_numpy(_columns(s, 6, 12).astype(np.float32)).cuda()
    Z = torch.zeros_like(R)
    nmg.check(nmg.nmg_vcycle_many(S.handle, solve_opts(precision=1), 6, R, Z))
    for k in (0, 5):
        z = torch.zeros_like(R[k])
        nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=1), R[k].contiguous(), z))
        assert torch.equal(Z[k], z)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("nrhs", [3, 9])
def test_solve_many_equals_single(nmg, built, sessions, case, prec, nrhs):
    s, h, _ = built[case]
    S = sessions[case]
    B = torch.from_numpy(_columns(s, nrhs, 13)).cuda()
    X = torch.full_like(B, float("nan"))
    infos = S.solve_many(B, X, nrhs, precision=prec)
    assert len(infos) == nrhs
    for k in range(nrhs):
        x = torch.empty_like(B[k])
        info = S.solve(B[k].contiguous(), x, precision=prec, use_graph=0, engine=nmg.NMG_ENGINE_KERNELS)
        assert infos[k].status == info.status == 0
        assert infos[k].iterations == info.iterations, (k, infos[k].iterations, info.iterations)
        assert torch.equal(X[k], x), k
    # every column reaches the method's tolerance on the oracle's operator
    for k in range(nrhs):
        b = B[k].cpu().numpy()
        xg = X[k].cpu().numpy()
        assert np.linalg.norm(b - h.fine.A.matvec(xg)) <= 1e-8 * np.linalg.norm(b)


def test_solve_many_matches_oracle_and_device_loop(nmg, built, sessions):
    """Column 0 (the workload's own right-hand side) against the oracle's FGMRES
    solution, and each column against the device-loop single solve."""
    s, h, _ = built["2d_32x32_3lev"]
    S = sessions["2d_32x32_3lev"]
    B = torch.from_numpy(_columns(s, 4, 14)).cuda()
    X = torch.zeros_like(B)
    infos = S.solve_many(B, X, 4, precision=1)
    xt, _ = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-11)
    xo, _ = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8)
    assert rel(X[0].cpu().numpy(), xt) <= max(1e-7, 20 * rel(xo, xt))
    for k in range(4):
        x = torch.empty_like(B[k])
        info = S.solve(B[k].contiguous(), x, precision=1, use_graph=2, engine=nmg.NMG_ENGINE_KERNELS)
        assert info.iterations == infos[k].iterations
        assert torch.equal(X[k], x)


def test_solve_many_host_buffers_and_zero_column(nmg, built, sessions):
    """Host b and x; a zero column finishes at once with x = 0 while the others
    iterate; a column that reaches maxit reports NOT_CONVERGED on its own."""
    s, _, _ = built["2d_24x40_3lev"]
    S = sessions["2d_24x40_3lev"]
    Bn = _columns(s, 5, 15)
    Bn[2] = 0.0
    Xn = np.full_like(Bn, np.nan)
    infos = S.solve_many(Bn, Xn, 5, precision=1)
    assert infos[2].status == 0 and infos[2].iterations == 0
    assert np.count_nonzero(Xn[2]) == 0
    Bd = torch.from_numpy(Bn).cuda()
    Xd = torch.zeros_like(Bd)
    infos_d = S.solve_many(Bd, Xd, 5, precision=1)
    for k in range(5):
        assert infos[k].iterations == infos_d[k].iterations
        assert np.array_equal(Xn[k], Xd[k].cpu().numpy())
    # maxit below what the columns need: every non-zero column stops unconverged,
    # with the status, count and iterate of the single solve
    infos_m = (nmg.nmg_solve_info * 5)()
    from paper_1904_02401_gb300.session import solve_opts
    st = nmg.nmg_solve_many(S.handle, 5, Bd, Xd, solve_opts(precision=1, maxit=2), infos_m)
    assert st == nmg.NMG_ERR_NOT_CONVERGED
    for k in range(5):
        x = torch.empty_like(Bd[k])
        info = S.solve(Bd[k].contiguous(), x, precision=1, maxit=2, use_graph=0, engine=nmg.NMG_ENGINE_KERNELS)
        assert infos_m[k].status == info.status == (0 if k == 2 else nmg.NMG_ERR_NOT_CONVERGED)
        assert infos_m[k].iterations == info.iterations
        assert torch.equal(Xd[k], x)


def test_many_refusals_and_bytes(nmg, built, sessions):
    from paper_1904_02401_gb300.session import solve_opts
    s, _, _ = built["2d_32x32_3lev"]
    S = sessions["2d_32x32_3lev"]
    R = torch.zeros(2, s.rhs.size, dtype=torch.float32, device="cuda")
    assert nmg.nmg_vcycle_many(S.handle, solve_opts(precision=1), 0, R, R.clone()) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_vcycle_many(S.handle, solve_opts(precision=0), 2, R, R.clone()) == nmg.NMG_ERR_INVALID
    B = torch.zeros(2, s.rhs.size, dtype=torch.float64, device="cuda")
    assert nmg.nmg_solve_many(S.handle, 2, B, B.clone(), solve_opts(precision=0)) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_solve_many(S.handle, 0, B, B.clone(), solve_opts(precision=1)) == nmg.NMG_ERR_INVALID
    # the column workspaces made by the multi-vector solves are counted
    before = S.bytes()
    B9 = torch.from_numpy(_columns(s, 8, 16)).cuda()
    S.solve_many(B9, torch.zeros_like(B9), 8, precision=1)
    assert S.bytes() >= before


@pytest.mark.parametrize("case", ["2d_24x40_3lev", "3d_8x12x16_3lev"])
@pytest.mark.parametrize("nu", [(0, 2), (1, 1), (2, 0), (3, 1)])
@pytest.mark.parametrize("weighting", [0, 1])
def test_vcycle_many_smoothing_variants(nmg, built, sessions, case, nu, weighting):
    """Other pre/post-smoothing counts (including none before or after), both
    overlap weightings and another damping: still equal to the single V-cycle
    per column bit for bit, plain launches and graph replay alike."""
    from paper_1904_02401_gb300.session import solve_opts
    s, _, _ = built[case]
    S = sessions[case]
    R = torch.from_numpy(_columns(s, 5, 17).astype(np.float32)).cuda()
    kw = dict(precision=1, nu1=nu[0], nu2=nu[1], weighting=weighting, omega=0.7)
    for graph in (0, 1):
        Z = torch.full_like(R, float("nan"))
        nmg.check(nmg.nmg_vcycle_many(S.handle, solve_opts(use_graph=graph, **kw), 5, R, Z))
        for k in (0, 4):
            z = torch.zeros_like(R[k])
            nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(use_graph=0, engine=nmg.NMG_ENGINE_KERNELS, **kw),
                                     R[k].contiguous(), z))
            assert torch.equal(Z[k], z), (graph, k)
