"""Degenerate and boundary cases of the C ABI on the GPU, checked against the oracle.

A zero right-hand side, a hierarchy of one level (the coarse direct solve
is the whole preconditioner), levels that hold exactly one patch, and mesh
descriptions the library must refuse.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import Problem, build_ale_system, build_system
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300 import nmg as lib
    return lib


def _session(s, ncomp=None):
    from paper_1904_02401_gb300.session import Session
    return Session(s.problem.dim, s.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet,
                   ncomp=ncomp)


def _dense(level):
    import scipy.sparse as sp
    nc = level.vals.shape[1]
    return sp.bsr_matrix((level.vals, level.col_idx, level.row_ptr), shape=(level.nodes * nc,) * 2).toarray()


def test_zero_rhs(nmg):
    s = build_system(Problem(dim=2, n=(16, 16), levels=3, solid=(0, +1, 0.6)))
    with _session(s) as S:
        b = torch.zeros(s.unknowns, dtype=torch.float64, device="cuda")
        x = torch.full_like(b, 3.0)
        for prec in (0, 1):
            info = S.solve(b, x, precision=prec)
            assert info.status == 0 and info.iterations == 0
            assert torch.count_nonzero(x).item() == 0


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
@pytest.mark.parametrize("engine", [0, 1])
def test_single_level_hierarchy(nmg, dim, n, engine):
    """One level: the V-cycle is the exact coarse solve, so FGMRES converges in
    one step to the dense solution."""
    p = Problem(dim=dim, n=(n,) * dim, levels=1, solid=(0, +1, 0.6) if dim == 2 else (2, -1, 0.25))
    s = build_system(p)
    xd = np.linalg.solve(_dense(s.fine), s.rhs)
    with _session(s) as S:
        b = torch.from_numpy(s.rhs).cuda()
        for prec in (0, 1):
            x = torch.empty_like(b)
            info = S.solve(b, x, precision=prec, engine=engine)
            assert info.status == 0
            assert info.iterations <= (1 if prec == 0 else 3)
            assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("dim", [2, 3])
def test_one_patch_level(nmg, dim):
    """Finest level of 2^d cells: a single Vanka patch covers it and the
    coarsest level is one cell.  The extension problem is used because it stays
    nonsingular on a mesh this small (the condensed momentum system without an
    interface leaves the pressure constant free).  The FP64 solve matches the
    oracle."""
    p = Problem(dim=dim, n=(2,) * dim, levels=2, solid=None)
    s = build_ale_system(p)
    h = Hierarchy(s.levels, s.dirichlet)
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8)
    with _session(s, ncomp=dim) as S:
        b = torch.from_numpy(s.rhs).cuda()
        x = torch.empty_like(b)
        info = S.solve(b, x, precision=0)
        assert info.status == 0
        assert abs(info.iterations - info_o["iterations"]) <= 1
        xg = x.cpu().numpy()
        if np.linalg.norm(xo) > 0:
            assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)


def test_refused_descriptions(nmg):
    """ncomp other than dim or dim + 1, no levels, cells not divisible by
    2^(levels - 1), a coarsest level beyond the dense solve: NMG_ERR_INVALID,
    nothing created."""
    mask = np.zeros(3 * 65 * 65, dtype=np.uint8)

    def create(dim=2, n=(8, 8), levels=2, ncomp=3):
        d = nmg.nmg_mesh_desc()
        d.dim = dim
        for k in range(3):
            d.n[k] = n[k] if k < dim else 1
        d.levels = levels
        d.ncomp = ncomp
        d.patch_cells = 2
        d.dirichlet_mask = mask.ctypes.data
        h = C.c_void_p()
        st = nmg.nmg_create_hierarchy(d, h)
        if st == 0:
            nmg.nmg_destroy_hierarchy(h)
        return st

    assert create() == 0
    assert create(ncomp=2) == 0            # n_c = d
    assert create(ncomp=4) == nmg.NMG_ERR_INVALID
    assert create(ncomp=1) == nmg.NMG_ERR_INVALID
    assert create(levels=0) == nmg.NMG_ERR_INVALID
    assert create(n=(12, 8), levels=4) == nmg.NMG_ERR_INVALID   # 12 not divisible by 8
    assert create(n=(6, 6), levels=2) == 0                     # coarsest level of 3 x 3 cells
    assert create(n=(12, 12), levels=2) == 0
    assert create(n=(64, 64), levels=1) == nmg.NMG_ERR_INVALID  # 65^2 x 3 unknowns on the coarsest level


@pytest.mark.parametrize("prec", [0, 1])
def test_bounded_barrier_wait_times_out_and_recovers(nmg, prec):
    """Every device-side wait is bounded.  With the persistent engine's grid-
    barrier limit set to one poll, the barriers of a V-cycle run out: the
    V-cycle and the solve return NMG_ERR_TIMEOUT without a fault, the flag is
    cleared, and with the default limit restored the same hierarchy solves
    again with exactly the result of a solve that never timed out."""
    from paper_1904_02401_gb300.session import solve_opts
    s = build_system(Problem(dim=2, n=(64, 64), levels=4, solid=(0, +1, 0.6)))
    S = _session(s)
    try:
        b = torch.from_numpy(s.rhs).cuda()
        o = solve_opts(precision=prec, engine=nmg.NMG_ENGINE_PERSISTENT, use_graph=0)
        ref = torch.empty_like(b)
        info = nmg.nmg_solve_info()
        assert nmg.nmg_solve(S.handle, b, ref, o, info) == nmg.NMG_OK
        its = info.iterations
        dt = torch.float64 if prec == 0 else torch.float32
        r = b.to(dt)
        z = torch.zeros_like(r)
        nmg.check(nmg.nmg_set_wait_limit(S.handle, 1))
        assert nmg.nmg_vcycle(S.handle, o, r, z) == nmg.NMG_ERR_TIMEOUT
        assert "aborted" in nmg.nmg_last_error()
        x = torch.empty_like(b)
        ot = solve_opts(precision=prec, engine=nmg.NMG_ENGINE_PERSISTENT, use_graph=0, maxit=40)
        assert nmg.nmg_solve(S.handle, b, x, ot, info) == nmg.NMG_ERR_TIMEOUT
        assert info.status == nmg.NMG_ERR_TIMEOUT
        nmg.check(nmg.nmg_set_wait_limit(S.handle, 0))
        assert nmg.nmg_solve(S.handle, b, x, o, info) == nmg.NMG_OK
        assert info.iterations == its
        assert torch.equal(x, ref)
        # the other engines never used the limit
        o2 = solve_opts(precision=prec, engine=nmg.NMG_ENGINE_KERNELS, use_graph=1)
        assert nmg.nmg_solve(S.handle, b, x, o2, info) == nmg.NMG_OK
    finally:
        S.close()
