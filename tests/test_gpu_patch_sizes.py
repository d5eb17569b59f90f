"""Vanka patches of two sizes on the GPU (nmg_set_large_patches; Section 5.5.1)
against the oracle with the same layout (oracle.multigrid.Hierarchy with
large_cells): the layout, the patch inverses of both sizes, one smoothing
step, the V-cycle and the solves, in FP64, FP32 and BF16.  Tolerances as in
the uniform-patch tests (tests/rounding_bounds.py)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import Problem, build_system
from gen.q1fsi import solid_cells
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy
from oracle.vanka import group_weights
from rounding_bounds import model_vcycle_dz, to_storage32, vanka_groups_step_and_bound, vcycle_tolerance, within

pytestmark = pytest.mark.gpu

CASES = {
    # large patches on the solid (interface on the coarsest grid line) or on every cell
    "2d_16_solid": (Problem(dim=2, n=(16, 16), levels=3, solid=(0, +1, 0.5)), "solid"),
    "2d_24x40_all": (Problem(dim=2, n=(24, 40), levels=3, solid=(0, +1, 0.6)), "all"),
    "2d_32_fluid": (Problem(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6)), "fluid"),
    "3d_8_solid": (Problem(dim=3, n=(8, 8, 8), levels=2, solid=(2, -1, 0.5)), "solid"),
    "3d_16_solid": (Problem(dim=3, n=(16, 16, 16), levels=3, solid=(2, -1, 0.25)), "solid"),
}


def _region(p, kind):
    solid = solid_cells(p, p.n)
    return {"solid": solid, "fluid": ~solid, "all": np.ones_like(solid)}[kind]


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300.session import Session
    out = {}
    for name, (p, kind) in CASES.items():
        s = build_system(p)
        region = _region(p, kind)
        h = Hierarchy(s.levels, s.dirichlet, large_cells=region)
        S = Session(p.dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet)
        S.set_large_patches(region)
        out[name] = (s, h, S)
    yield out
    for _, _, S in out.values():
        S.close()


def _groups(L):
    return L.groups if L.groups is not None else [(L.dofs, L.Ainv)]


@pytest.mark.parametrize("case", list(CASES))
def test_layout_and_inverses(built, case):
    from paper_1904_02401_gb300 import nmg
    s, h, S = built[case]
    nlarge_total = 0
    for lev in range(1, len(h.levels)):
        L = h.levels[lev]
        groups = _groups(L)
        ns_o = groups[0][0].shape[0] if groups[0][0].shape[1] == S.patch_layout(lev)[2] else 0
        nl_o = sum(g[0].shape[0] for g in groups if g[0].shape[1] != S.patch_layout(lev)[2])
        ns, nl, ps, pl = S.patch_layout(lev)
        assert (ns, nl) == (ns_o, nl_o), (lev, ns, nl, ns_o, nl_o)
        nlarge_total += nl
        # sampled inverses of both sizes, in the oracle's order (small, then large)
        for prec in (0, 1, 2):
            for k0, (dofs, inv) in zip((0, ns), [(g[0], g[1]) for g in groups]):
                n_p = dofs.shape[1]
                for k in sorted({0, inv.shape[0] - 1, inv.shape[0] // 2}):
                    out = np.empty((1, n_p, n_p))
                    nmg.check(nmg.nmg_get_patch_inverses(S.handle, lev, prec, k0 + k, 1, out))
                    ref = inv[k]
                    m = np.abs(ref).max()
                    rel = {0: 0.0, 1: 2.0 ** -23, 2: 2.0 ** -8}[prec]
                    assert np.all(np.abs(out[0] - ref) <= rel * np.abs(ref) + 1e-7 * m), (lev, prec, k)
    assert nlarge_total > 0
    # a range across both sizes is refused
    lev = len(h.levels) - 1
    ns, nl, ps, pl = S.patch_layout(lev)
    if ns and nl:
        out = np.empty((2, pl, pl))
        assert nmg.nmg_get_patch_inverses(S.handle, lev, 0, ns - 1, 2, out) == nmg.NMG_ERR_INVALID


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("weighting", [0, 1])
def test_one_smoothing_step(built, case, prec, weighting):
    from paper_1904_02401_gb300 import nmg
    s, h, S = built[case]
    dim, nc = s.problem.dim, s.problem.ncomp
    omega = 0.8 if weighting == 0 else 0.3
    rng = np.random.default_rng(13)
    dt = torch.float64 if prec == 0 else torch.float32
    for lev in range(1, len(h.levels)):
        L = h.levels[lev]
        groups = _groups(L)
        n = L.A.size
        b = to_storage32(rng.uniform(-1, 1, n))
        x0 = to_storage32(rng.uniform(-1, 1, n))
        d = b - L.A.matvec(x0)
        w = group_weights(groups, n, "average" if weighting == 0 else "sum")
        xd = torch.from_numpy(x0).to(dt).cuda()
        nmg.check(nmg.nmg_smooth(S.handle, lev, prec, torch.from_numpy(b).to(dt).cuda(), xd, 1, 0, omega, weighting))
        got = xd.double().cpu().numpy()
        if prec == 0:
            ref = x0 + omega * w * sum(_corr(g, d, n) for g in groups)
            assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), lev
        else:
            ref, bound = vanka_groups_step_and_bound(groups, b, x0, d, abs(L.A.csr) @ np.abs(x0), w, omega, prec,
                                                     dim, nc)
            assert np.all(np.abs(got - ref) <= bound), (lev, (np.abs(got - ref) / (bound + 1e-300)).max())


def _corr(group, d, n):
    dofs, inv = group
    c = np.zeros(n)
    np.add.at(c, dofs, np.einsum("pij,pj->pi", inv, d[dofs]))
    return c


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_vcycle(built, case, prec, use_graph):
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    s, h, S = built[case]
    nc = s.problem.ncomp
    r = to_storage32(s.rhs)
    dt = torch.float64 if prec == 0 else torch.float32
    z = torch.zeros(r.size, dtype=dt, device="cuda")
    nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=use_graph), torch.from_numpy(r).to(dt).cuda(),
                             z))
    err = z.double().cpu().numpy()
    if prec == 0:
        ref = h.vcycle(r)
        assert np.abs(err - ref).max() <= 1e-8 * np.abs(ref).max()
    else:
        dz, ref = model_vcycle_dz(h, r, {1: "fp32", 2: "bf16"}[prec], nc)
        tol = vcycle_tolerance(dz, np.abs(ref).max(), nc)
        assert within(err - ref, tol, nc).all(), (np.abs(err - ref).reshape(-1, nc).max(0), tol)


@pytest.mark.parametrize("case", list(CASES))
def test_solves(built, case):
    """FP64: equal iteration counts (tie rule) and solution within 1e-8 of the
    oracle's; FP32 / BF16: true FP64 residual <= 1e-8."""
    s, h, S = built[case]
    hist = []
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8, history=hist)
    b = torch.from_numpy(s.rhs).cuda()
    for prec in (0, 1, 2):
        x = torch.empty_like(b)
        info = S.solve(b, x, precision=prec)
        assert info.status == 0 and info.engine == 1
        xg = x.cpu().numpy()
        assert np.linalg.norm(s.rhs - h.fine.A.matvec(xg)) <= 1e-8 * np.linalg.norm(s.rhs)
        if prec == 0:
            near = any(1e-8 / 1.01 <= v <= 1e-8 * 1.01 for v in hist[-2:])
            assert info.iterations == info_o["iterations"] or (near and abs(info.iterations - info_o["iterations"]) <= 1)
            assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)


def test_refusals_and_reset(built):
    """Other engines and multi-vector calls are refused with patches of two
    sizes; a NULL mask restores the single size and its results."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import Session, solve_opts
    s, h, S = built["2d_16_solid"]
    b = torch.from_numpy(s.rhs).cuda()
    x = torch.empty_like(b)
    for eng in (nmg.NMG_ENGINE_PERSISTENT, nmg.NMG_ENGINE_FUSED):
        assert nmg.nmg_solve(S.handle, b, x, solve_opts(engine=eng), nmg.nmg_solve_info()) == nmg.NMG_ERR_INVALID
    r = torch.zeros((2, s.unknowns), dtype=torch.float32, device="cuda")
    assert nmg.nmg_vcycle_many(S.handle, solve_opts(precision=1), 2, r, torch.zeros_like(r)) == nmg.NMG_ERR_INVALID
    p = s.problem
    with Session(p.dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet) as T:
        T.set_large_patches(_region(p, "solid"))
        T.set_large_patches(None)
        assert T.patch_layout(len(s.levels) - 1)[1] == 0
        x1, x2 = torch.empty_like(b), torch.empty_like(b)
        with Session(p.dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet) as U:
            o = solve_opts(precision=1, engine=nmg.NMG_ENGINE_KERNELS, use_graph=1)
            T.solve(b, x1, **{k: getattr(o, k) for k in ("precision", "engine", "use_graph")})
            U.solve(b, x2, **{k: getattr(o, k) for k in ("precision", "engine", "use_graph")})
        assert torch.equal(x1, x2)
