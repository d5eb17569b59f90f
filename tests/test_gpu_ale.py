"""GPU parity of the ALE-extension solve (problem (3) of Section 4.2, n_c = d).

The same library (hierarchy, block products, Vanka patch inversion and
smoothing, transfers, coarse solve, FGMRES) runs the d-component harmonic
extension with patches of 3^d nodes x d unknowns (18 in 2d, 81 in 3d).  Every
step is compared with the FP64 CPU oracle on the same seeded inputs, and the
full solves with the oracle's FGMRES.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import Problem, build_ale_system
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy

pytestmark = pytest.mark.gpu

CASES = {
    "ale_2d_32x32_3lev": Problem(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6)),
    "ale_2d_24x40_3lev": Problem(dim=2, n=(24, 40), levels=3, solid=(0, +1, 0.6)),
    "ale_3d_8x12x16_3lev": Problem(dim=3, n=(8, 12, 16), levels=3, solid=(2, -1, 0.5)),
    "ale_3d_16_3lev": Problem(dim=3, n=(16, 16, 16), levels=3, solid=(2, -1, 0.25)),
}
PRECS = [0, 1, 2]


@pytest.fixture(scope="module")
def nmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300 import nmg as lib
    return lib


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, p in CASES.items():
        s = build_ale_system(p)
        out[name] = (s, Hierarchy(s.levels, s.dirichlet))
    return out


@pytest.fixture(scope="module")
def sessions(nmg, built):
    from paper_1904_02401_gb300.session import Session
    out = {}
    for name, (s, _) in built.items():
        out[name] = Session(s.problem.dim, s.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels],
                            s.dirichlet, ncomp=s.problem.dim)
    yield out
    for v in out.values():
        v.close()


def cu(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def vdtype(prec):
    return np.float64 if prec == 0 else np.float32


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_ale_matvec_and_residual(nmg, built, sessions, case, prec):
    s, h = built[case]
    S = sessions[case]
    rng = np.random.default_rng(7)
    dt = vdtype(prec)
    tol = 1e-13 if prec == 0 else 1e-5
    for lev, L in enumerate(h.levels):
        n = L.A.size
        x = rng.standard_normal(n).astype(dt).astype(np.float64)
        b = rng.standard_normal(n).astype(dt).astype(np.float64)
        xd, bd = cu(x, dt), cu(b, dt)
        y = torch.empty_like(xd)
        nmg.check(nmg.nmg_matvec(S.handle, lev, prec, xd, y))
        A = L.A.csr
        Avals = A.astype(dt).astype(np.float64) if prec else A
        ref = Avals @ x
        scale = abs(Avals) @ abs(x) + 1e-300
        assert np.max(np.abs(host(y) - ref) / scale) < tol
        nmg.check(nmg.nmg_residual(S.handle, lev, prec, bd, xd, y))
        assert np.max(np.abs(host(y) - (b - ref)) / (scale + abs(b))) < tol


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_ale_patch_inverses(nmg, built, sessions, case, prec):
    s, h = built[case]
    S = sessions[case]
    for lev in range(1, len(h.levels)):
        L = h.levels[lev]
        P, npd = L.Ainv.shape[0], L.Ainv.shape[1]
        assert npd == (9 if s.problem.dim == 2 else 27) * s.problem.dim
        for first in sorted({0, 1, P // 2, P - 1}):
            out = np.empty((1, npd, npd))
            nmg.check(nmg.nmg_get_patch_inverses(S.handle, lev, prec, first, 1, out))
            ref = L.Ainv[first]
            tol = 1e-12 if prec == 0 else (1e-6 if prec == 1 else 1e-2)
            assert np.abs(out[0] - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("weighting", [0, 1])
def test_ale_vanka_smoothing(nmg, built, sessions, case, prec, weighting):
    from oracle.vanka import overlap_weights, vanka_step
    s, h = built[case]
    S = sessions[case]
    dt = vdtype(prec)
    rng = np.random.default_rng(3)
    om = 0.8 if weighting == 0 else 0.3
    for lev in range(1, len(h.levels)):
        L = h.levels[lev]
        n = L.A.size
        b = rng.standard_normal(n).astype(dt).astype(np.float64)
        x0 = rng.standard_normal(n).astype(dt).astype(np.float64)
        wgt = overlap_weights(L.dofs, n, "average" if weighting == 0 else "sum")
        for x_zero in (1, 0):
            ref = np.zeros(n) if x_zero else x0
            for _ in range(2):
                ref = vanka_step(L.A, L.Ainv, L.dofs, b, ref, om, wgt)
            xd = cu(x0, dt)
            nmg.check(nmg.nmg_smooth(S.handle, lev, prec, cu(b, dt), xd, 2, x_zero, om, weighting))
            tol = 1e-8 if prec == 0 else (1e-4 if prec == 1 else 3e-2)
            assert rel(host(xd), ref) < tol, (lev, x_zero)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_ale_transfers_and_coarse(nmg, built, sessions, case, prec):
    s, h = built[case]
    S = sessions[case]
    dt = vdtype(prec)
    rng = np.random.default_rng(5)
    tol = 1e-14 if prec == 0 else 1e-6
    for lev in range(1, len(h.levels)):
        Lf, Lc = h.levels[lev], h.levels[lev - 1]
        r = rng.standard_normal(Lf.A.size).astype(dt).astype(np.float64)
        rc = torch.zeros(Lc.A.size, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        nmg.check(nmg.nmg_restrict(S.handle, lev, prec, cu(r, dt), rc))
        ref = Lf.P.T @ r
        ref[Lc.mask] = 0.0
        assert np.abs(host(rc) - ref).max() <= tol * np.abs(ref).max()
        e = rng.standard_normal(Lc.A.size).astype(dt).astype(np.float64)
        x = rng.standard_normal(Lf.A.size).astype(dt).astype(np.float64)
        xd = cu(x, dt)
        nmg.check(nmg.nmg_prolongate_add(S.handle, lev, prec, cu(e, dt), xd))
        corr = Lf.P @ e
        corr[Lf.mask] = 0.0
        assert np.abs(host(xd) - (x + corr)).max() <= 4 * tol * np.abs(x + corr).max()
    b = rng.standard_normal(h.levels[0].A.size).astype(dt).astype(np.float64)
    xd = torch.zeros(b.size, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    nmg.check(nmg.nmg_coarse_solve(S.handle, prec, cu(b, dt), xd))
    assert rel(host(xd), h.coarse_solve(b)) < (1e-8 if prec == 0 else 1e-5)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_ale_solve_fp64_matches_oracle(nmg, built, sessions, case, use_graph):
    s, h = built[case]
    S = sessions[case]
    hist = []
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8, history=hist)
    b = cu(s.rhs, np.float64)
    x = torch.empty_like(b)
    info = S.solve(b, x, precision=0, use_graph=use_graph)
    assert info.status == 0
    # equal counts; one either way only when the final estimate lies within 1 % of rtol
    near = any(1e-8 / 1.01 <= v <= 1e-8 * 1.01 for v in hist[-2:])
    assert info.iterations == info_o["iterations"] or (near and abs(info.iterations - info_o["iterations"]) <= 1), \
        (info.iterations, info_o)
    xg = host(x)
    assert rel(xg, xo) <= 1e-8
    assert np.linalg.norm(s.rhs - h.fine.A.matvec(xg)) / np.linalg.norm(s.rhs) <= 1e-8


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [1, 2])
def test_ale_solve_mixed_precision(nmg, built, sessions, case, prec):
    s, h = built[case]
    S = sessions[case]
    b = cu(s.rhs, np.float64)
    x = torch.empty_like(b)
    info = S.solve(b, x, precision=prec)
    assert info.status == 0
    xg = host(x)
    relres = np.linalg.norm(s.rhs - h.fine.A.matvec(xg)) / np.linalg.norm(s.rhs)
    assert relres <= 1e-8
    xt, _ = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-11)
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8)
    assert rel(xg, xt) <= max(1e-7, 20 * rel(xo, xt))
    assert info.iterations <= info_o["iterations"] + 3


def test_ale_engines(nmg, built, sessions):
    """n_c = d hierarchies run the per-step engine (plain, graph and device
    loop agree bitwise); the persistent and fused engines are refused."""
    from paper_1904_02401_gb300.session import solve_opts
    s, h = built["ale_2d_32x32_3lev"]
    S = sessions["ale_2d_32x32_3lev"]
    r = cu(s.rhs.astype(np.float32), np.float32)
    outs = []
    for graph in (0, 1):
        for engine in (nmg.NMG_ENGINE_AUTO, nmg.NMG_ENGINE_KERNELS):
            z = torch.zeros_like(r)
            nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=1, use_graph=graph, engine=engine), r, z))
            outs.append(z)
    for z in outs[1:]:
        assert torch.equal(z, outs[0])
    for engine in (nmg.NMG_ENGINE_PERSISTENT, nmg.NMG_ENGINE_FUSED):
        z = torch.zeros_like(r)
        assert nmg.nmg_vcycle(S.handle, solve_opts(precision=1, engine=engine), r, z) == nmg.NMG_ERR_INVALID
