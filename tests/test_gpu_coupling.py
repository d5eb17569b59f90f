"""Problems (2) and (3) of Section 4.2 on the GPU, against the oracle's
sub-steps (oracle/coupling.py, pinned to the monolithic block solve in
tests/test_coupling_pins.py): the deformation update, the lifting of the fixed
values into the extension's right-hand side, and the whole chain
nmg_newton_substeps (momentum solve, deformation update, extension solve)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import Problem, build_ale_system, build_system
from gen.q1fsi import _dirichlet_nodes, ale_fixed_nodes, assemble_ale_level, solid_cells
from oracle.bsr import BlockMatrix
from oracle.coupling import deformation_update, extension_rhs, linear_newton_step
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy

pytestmark = pytest.mark.gpu

K_THETA = 0.01
CASES = {
    "2d_32_3lev": Problem(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6)),
    "2d_24x40_3lev": Problem(dim=2, n=(24, 40), levels=3, solid=(0, +1, 0.6)),
    "3d_8_2lev": Problem(dim=3, n=(8, 8, 8), levels=2, solid=(2, -1, 0.5)),
    "3d_16_3lev": Problem(dim=3, n=(16, 16, 16), levels=3, solid=(2, -1, 0.25)),
}


@pytest.fixture(scope="module")
def nmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300 import nmg as lib
    return lib


def _setup(p):
    """Both systems of the mesh, the unreduced extension operator, the node
    sets (fixed = solid-cell nodes and boundary; update = solid-cell nodes off
    the boundary) and seeded r (zero off the update nodes) and b5."""
    s1, s3 = build_system(p), build_ale_system(p)
    Ef = assemble_ale_level(p, p.n, eliminate=False)
    solid = solid_cells(p, p.n)
    fixed = ale_fixed_nodes(p.dim, p.n, solid).reshape(-1)
    update = fixed & ~_dirichlet_nodes(p.dim, p.n).reshape(-1)
    rng = np.random.default_rng(61)
    nodes = fixed.size
    r = rng.uniform(-1, 1, nodes * p.dim)
    r.reshape(nodes, p.dim)[~update] = 0.0
    b5 = rng.uniform(-1, 1, nodes * p.dim)
    return s1, s3, Ef, fixed, update, r, b5


def _sessions(nmg, p, s1, s3, Ef):
    from paper_1904_02401_gb300.session import Session
    S1 = Session(p.dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in s1.levels], s1.dirichlet)
    S3 = Session(p.dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in s3.levels], s3.dirichlet, ncomp=p.dim)
    nmg.check(nmg.nmg_set_lifting_operator(S3.handle, Ef.nodes, Ef.col_idx.size,
                                           np.ascontiguousarray(Ef.row_ptr, dtype=np.int64),
                                           np.ascontiguousarray(Ef.col_idx, dtype=np.int32),
                                           np.ascontiguousarray(Ef.vals, dtype=np.float64), 0))
    return S1, S3


def _cu(a, dt=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


@pytest.mark.parametrize("case", list(CASES))
def test_deformation_update_and_lifting(nmg, case):
    p = CASES[case]
    s1, s3, Ef, fixed, update, r, b5 = _setup(p)
    S1, S3 = _sessions(nmg, p, s1, s3, Ef)
    try:
        nodes = fixed.size
        dv = np.random.default_rng(62).uniform(-1, 1, nodes * (p.dim + 1))
        du = torch.full((nodes * p.dim,), float("nan"), dtype=torch.float64, device="cuda")
        nmg.check(nmg.nmg_deformation_update(S3.handle, _cu(r), _cu(dv), K_THETA, _cu(update, np.uint8), du))
        ref = deformation_update(r, dv, K_THETA, update, p.dim)
        got = du.cpu().numpy()
        assert np.abs(got - ref).max() <= 2.0 ** -50 * np.abs(ref).max()   # a fused multiply-add either way
        assert np.count_nonzero(got.reshape(nodes, p.dim)[~update]) == 0
        # the lifting: g = that deformation on the fixed nodes
        E = BlockMatrix(Ef.row_ptr, Ef.col_idx, Ef.vals)
        rhs = torch.full_like(du, float("nan"))
        nmg.check(nmg.nmg_extension_rhs(S3.handle, _cu(b5), du, rhs))
        ref = extension_rhs(E, b5, fixed, ref, p.dim)
        F = np.repeat(fixed, p.dim)
        ghat = np.where(F, got, 0.0)
        scale = np.abs(b5) + abs(E.csr) @ np.abs(ghat)
        out = rhs.cpu().numpy()
        assert np.array_equal(out[F], got[F])
        assert np.all(np.abs(out - ref) <= 1e-14 * scale + 1e-300)
    finally:
        S1.close()
        S3.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("host", [False, True])
def test_newton_substeps_match_the_oracle(nmg, case, host):
    """FP64 solves: both solutions within 1e-8 of the oracle's sub-steps (FGMRES
    with the oracle's V-cycle at the same rtol), iteration counts equal (one
    either way when the estimate ends within 1 % of rtol)."""
    from paper_1904_02401_gb300.session import solve_opts
    p = CASES[case]
    s1, s3, Ef, fixed, update, r, b5 = _setup(p)
    S1, S3 = _sessions(nmg, p, s1, s3, Ef)
    try:
        h1 = Hierarchy(s1.levels, s1.dirichlet)
        h3 = Hierarchy(s3.levels, s3.dirichlet)
        its = {}

        def solver(h, key):
            def f(b):
                hist = []
                x, info = fgmres(h.fine.A.matvec, h.vcycle, b, rtol=1e-8, history=hist)
                its[key] = (info["iterations"], hist)
                return x
            return f

        E = BlockMatrix(Ef.row_ptr, Ef.col_idx, Ef.vals)
        w_o, u_o = linear_newton_step(solver(h1, 1), s1.rhs, r, K_THETA, update, solver(h3, 3), E, b5, fixed, p.dim)
        nodes = fixed.size
        if host:
            b1, rr, bb5, upd = s1.rhs.copy(), r.copy(), b5.copy(), update.astype(np.uint8)
            dw, du = np.zeros(nodes * (p.dim + 1)), np.zeros(nodes * p.dim)
        else:
            b1, rr, bb5, upd = _cu(s1.rhs), _cu(r), _cu(b5), _cu(update, np.uint8)
            dw = torch.zeros(nodes * (p.dim + 1), dtype=torch.float64, device="cuda")
            du = torch.zeros(nodes * p.dim, dtype=torch.float64, device="cuda")
        i1, i3 = nmg.nmg_solve_info(), nmg.nmg_solve_info()
        o = solve_opts(precision=0)
        assert nmg.nmg_newton_substeps(S1.handle, S3.handle, b1, rr, K_THETA, upd, bb5, dw, du, o, o, i1, i3) == 0
        dw = dw if host else dw.cpu().numpy()
        du = du if host else du.cpu().numpy()
        for (gpu_its, key) in ((i1.iterations, 1), (i3.iterations, 3)):
            ora, hist = its[key]
            near = any(1e-8 / 1.01 <= v <= 1e-8 * 1.01 for v in hist[-2:])
            assert gpu_its == ora or (near and abs(gpu_its - ora) <= 1), (key, gpu_its, ora)
        assert np.linalg.norm(dw - w_o) <= 1e-8 * np.linalg.norm(w_o)
        assert np.linalg.norm(du - u_o) <= 1e-8 * np.linalg.norm(u_o)
        # on the fixed nodes the extension's solution is problem (2)'s deformation of this dw
        # (the identity rows hold to the solve's residual)
        F = np.repeat(fixed, p.dim)
        d2 = deformation_update(r, dw, K_THETA, update, p.dim)
        rhs3 = extension_rhs(E, b5, fixed, d2, p.dim)
        assert np.linalg.norm(du[F] - d2[F]) <= 1.01e-8 * np.linalg.norm(rhs3)
    finally:
        S1.close()
        S3.close()


@pytest.mark.parametrize("case", ["2d_32_3lev", "3d_16_3lev"])
@pytest.mark.parametrize("prec", [1, 2])
def test_newton_substeps_mixed_precision(nmg, case, prec):
    """Reduced-precision V-cycles in both solves: the true FP64 residuals of
    problems (1) and (3) reach 1e-8 and the results lie within 1e-6 of the
    FP64 chain's."""
    from paper_1904_02401_gb300.session import solve_opts
    p = CASES[case]
    s1, s3, Ef, fixed, update, r, b5 = _setup(p)
    S1, S3 = _sessions(nmg, p, s1, s3, Ef)
    try:
        nodes = fixed.size
        outs = []
        for pr in (0, prec):
            dw = torch.zeros(nodes * (p.dim + 1), dtype=torch.float64, device="cuda")
            du = torch.zeros(nodes * p.dim, dtype=torch.float64, device="cuda")
            o = solve_opts(precision=pr)
            nmg.check(nmg.nmg_newton_substeps(S1.handle, S3.handle, _cu(s1.rhs), _cu(r), K_THETA,
                                              _cu(update, np.uint8), _cu(b5), dw, du, o, o, None, None))
            outs.append((dw.cpu().numpy(), du.cpu().numpy()))
        (w0, u0), (w1, u1) = outs
        A1 = BlockMatrix(s1.fine.row_ptr, s1.fine.col_idx, s1.fine.vals)
        assert np.linalg.norm(s1.rhs - A1.matvec(w1)) <= 1e-8 * np.linalg.norm(s1.rhs)
        assert np.linalg.norm(w1 - w0) <= 1e-6 * np.linalg.norm(w0)
        assert np.linalg.norm(u1 - u0) <= 1e-6 * np.linalg.norm(u0)
    finally:
        S1.close()
        S3.close()


def test_substeps_refuse_mismatched_hierarchies(nmg):
    from paper_1904_02401_gb300.session import solve_opts
    p = CASES["2d_32_3lev"]
    s1, s3, Ef, fixed, update, r, b5 = _setup(p)
    S1, S3 = _sessions(nmg, p, s1, s3, Ef)
    try:
        o = solve_opts(precision=0)
        z = torch.zeros(s1.unknowns, dtype=torch.float64, device="cuda")
        z3 = torch.zeros(s3.unknowns, dtype=torch.float64, device="cuda")
        # the roles swapped: h3 must have ncomp = dim
        assert nmg.nmg_newton_substeps(S3.handle, S1.handle, z, z3, K_THETA, _cu(update, np.uint8), z3, z, z3, o, o,
                                       None, None) == nmg.NMG_ERR_INVALID
        assert nmg.nmg_set_lifting_operator(S1.handle, 1, 0, np.zeros(2, np.int64), None, None, 0) == \
            nmg.NMG_ERR_INVALID
        assert nmg.nmg_extension_rhs(S1.handle, z, z, z) == nmg.NMG_ERR_INVALID
    finally:
        S1.close()
        S3.close()
