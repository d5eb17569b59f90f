"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (derived from the arithmetic):
* FP64 block products: each output sums <= 27 * 4 products, so the error is
  below 1e-13 of sum |a||x| (108 * 2^-53 = 1.2e-14, with margin).
* FP32 block products: the same bound in float, 1e-5 of sum |a||x|.
* FP64 patch inverses: Gauss-Jordan and LAPACK getri differ by about
  kappa(A_i) * 2^-53; with kappa(A_i) <= ~1e8 here, 1e-7 of max |A_i^-1|.
* FP32 / BF16 stored inverses: one rounding of the FP64 inverse,
  2^-24 resp. 2^-8 relative per entry (plus the FP64 part).
* FP32 / BF16 smoothing and V-cycles: entry by entry, 8x the per-component
  deviation of the oracle run the binary32 way (binary32 matrices, vectors and
  arithmetic, inverses rounded to the storage format) plus 16 u times the
  largest entry (tests/rounding_bounds.py).
* FP64 smoother, V-cycle and solve: the patch-inverse differences propagate
  linearly, 1e-8 relative (the solve's bound is the one the method states:
  solution relative error <= 1e-8 with equal iteration counts).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import Problem, build_system
from oracle.bsr import BlockMatrix
from oracle.multigrid import Hierarchy
from oracle.fgmres import fgmres

pytestmark = pytest.mark.gpu

CASES = {
    "2d_32x32_3lev": Problem(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6)),
    "2d_24x40_3lev": Problem(dim=2, n=(24, 40), levels=3, solid=(0, +1, 0.6)),
    "3d_8_2lev": Problem(dim=3, n=(8, 8, 8), levels=2, solid=(2, -1, 0.25)),
    "3d_8x12x16_3lev": Problem(dim=3, n=(8, 12, 16), levels=3, solid=(2, -1, 0.5)),
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
        s = build_system(p)
        h = Hierarchy(s.levels, s.dirichlet)
        out[name] = (s, h)
    return out


@pytest.fixture(scope="module")
def sessions(nmg, built):
    from paper_1904_02401_gb300.session import Session
    out = {}
    for name, (s, _) in built.items():
        out[name] = Session(s.problem.dim, s.problem.n,
                            [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet)
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
def test_matvec_and_residual(nmg, built, sessions, case, prec):
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
        ref_r = b - ref
        scale_r = scale + abs(b)
        assert np.max(np.abs(host(y) - ref_r) / scale_r) < tol


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_patch_inverses(nmg, built, sessions, case, prec):
    s, h = built[case]
    S = sessions[case]
    for lev in range(1, len(h.levels)):
        L = h.levels[lev]
        P = L.Ainv.shape[0]
        npd = L.Ainv.shape[1]
        idx = sorted(set(list(range(min(P, 48))) + [P - 1, P // 2]))
        for first in idx:
            out = np.empty((1, npd, npd))
            nmg.check(nmg.nmg_get_patch_inverses(S.handle, lev, prec, first, 1, out))
            ref = L.Ainv[first]
            m = np.abs(ref).max()
            if prec == 0:
                assert np.abs(out[0] - ref).max() <= 1e-7 * m
            elif prec == 1:
                assert np.all(np.abs(out[0] - ref) <= 2.0 ** -23 * np.abs(ref) + 1e-7 * m)
            else:
                assert np.all(np.abs(out[0] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-7 * m)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("weighting", [0, 1])
def test_vanka_smoothing(nmg, built, sessions, case, prec, weighting):
    """Two steps of Eq. (vanka) on every smoothed level, from zero and from a
    random iterate, entry by entry: FP64 within 1e-8 of the largest entry;
    FP32 / BF16 within the per-component tolerance of tests/rounding_bounds.py
    (8x the deviation of the binary32 model of the steps, plus 16 u max|x|)."""
    from oracle.precision import with_fp32_arithmetic
    from oracle.vanka import overlap_weights, vanka_step
    from rounding_bounds import vcycle_tolerance, within
    s, h = built[case]
    S = sessions[case]
    dt = vdtype(prec)
    nc = s.problem.ncomp
    om = 0.8 if weighting == 0 else 0.3
    rng = np.random.default_rng(3)
    for lev in range(1, len(h.levels)):
        L = h.levels[lev]
        n = L.A.size
        b = rng.standard_normal(n).astype(dt).astype(np.float64)
        x0 = rng.standard_normal(n).astype(dt).astype(np.float64)
        wgt = overlap_weights(L.dofs, n, "average" if weighting == 0 else "sum")
        Lm = with_fp32_arithmetic(h, {1: "fp32", 2: "bf16"}[prec]).levels[lev] if prec else None
        for x_zero in (1, 0):
            ref = np.zeros(n) if x_zero else x0
            rs = ref.astype(np.float32)
            for _ in range(2):
                ref = vanka_step(L.A, L.Ainv, L.dofs, b, ref, om, wgt)
                if prec:
                    rs = vanka_step(Lm.A, Lm.Ainv, L.dofs, b.astype(np.float32), rs, np.float32(om),
                                    wgt.astype(np.float32))
            xd = cu(x0, dt)
            nmg.check(nmg.nmg_smooth(S.handle, lev, prec, cu(b, dt), xd, 2, x_zero, om, weighting))
            err = host(xd) - ref
            if prec == 0:
                assert np.abs(err).max() <= 1e-8 * np.abs(ref).max(), (lev, x_zero)
            else:
                tol = vcycle_tolerance(np.abs(rs - ref).reshape(-1, nc).max(axis=0), np.abs(ref).max(), nc)
                assert within(err, tol, nc).all(), (lev, x_zero, np.abs(err).reshape(-1, nc).max(0), tol)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_transfers_and_coarse(nmg, built, sessions, case, prec):
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
        c = Lf.P @ e
        c[Lf.mask] = 0.0
        ref = x + c
        assert np.abs(host(xd) - ref).max() <= 4 * tol * np.abs(ref).max()
    b = rng.standard_normal(h.levels[0].A.size).astype(dt).astype(np.float64)
    xd = torch.zeros(b.size, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    nmg.check(nmg.nmg_coarse_solve(S.handle, prec, cu(b, dt), xd))
    ref = h.coarse_solve(b)
    assert rel(host(xd), ref) < (1e-8 if prec == 0 else 1e-5)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("engine,use_graph", [(1, 0), (1, 1), (2, 0), (3, 0), (3, 1)])
def test_vcycle(nmg, built, sessions, case, prec, engine, use_graph):
    """One V(2,2) cycle entry by entry: FP64 within 1e-8 of the largest entry;
    FP32 / BF16 within 8x the per-component deviation of the binary32 model of
    the cycle plus 16 u max|z| (tests/rounding_bounds.py)."""
    from paper_1904_02401_gb300.session import solve_opts
    from rounding_bounds import model_vcycle_dz, vcycle_tolerance, within
    s, h = built[case]
    S = sessions[case]
    dt = vdtype(prec)
    nc = s.problem.ncomp
    r = s.rhs.astype(dt).astype(np.float64)
    z = torch.zeros(r.size, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=use_graph, engine=engine), cu(r, dt), z))
    ref = h.vcycle(r)
    err = host(z) - ref
    if prec == 0:
        assert np.abs(err).max() <= 1e-8 * np.abs(ref).max()
    else:
        dz, _ = model_vcycle_dz(h, r, {1: "fp32", 2: "bf16"}[prec], nc)
        tol = vcycle_tolerance(dz, np.abs(ref).max(), nc)
        assert within(err, tol, nc).all(), (np.abs(err).reshape(-1, nc).max(0), tol)


def _iteration_tie_ok(gpu_its, ora_its, hist, rtol):
    if gpu_its == ora_its:
        return True
    # the estimate crossed rtol within a factor 1.01: one step either way is accepted
    near = any(abs(v / rtol - 1.0) < 0.01 or (rtol / 1.01 <= v <= rtol * 1.01) for v in hist[-2:])
    return near and abs(gpu_its - ora_its) <= 1


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_solve_fp64_matches_oracle(nmg, built, sessions, case, use_graph):
    s, h = built[case]
    S = sessions[case]
    hist = []
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8, history=hist)
    b = cu(s.rhs, np.float64)
    x = torch.empty_like(b)
    info = S.solve(b, x, precision=0, use_graph=use_graph)
    assert info.status == 0
    assert info.device_loop == (1 if use_graph == 2 else 0)
    assert _iteration_tie_ok(info.iterations, info_o["iterations"], hist, 1e-8), (info.iterations, info_o)
    xg = host(x)
    assert rel(xg, xo) <= 1e-8
    assert np.linalg.norm(s.rhs - h.fine.A.matvec(xg)) / np.linalg.norm(s.rhs) <= 1e-8


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [1, 2])
def test_solve_mixed_precision(nmg, built, sessions, case, prec):
    s, h = built[case]
    S = sessions[case]
    b = cu(s.rhs, np.float64)
    x = torch.empty_like(b)
    info = S.solve(b, x, precision=prec)
    assert info.status == 0
    xg = host(x)
    relres = np.linalg.norm(s.rhs - h.fine.A.matvec(xg)) / np.linalg.norm(s.rhs)
    assert relres <= 1e-8
    assert abs(info.rel_residual - relres) <= 1e-3 * relres + 1e-15
    # forward error against a tightly converged FP64 oracle solve
    xt, _ = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-11)
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8)
    err = rel(xg, xt)
    err_o = rel(xo, xt)
    assert err <= max(1e-7, 20 * err_o), (err, err_o)
    assert info.iterations <= info_o["iterations"] + 3


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("restart,maxit", [(30, 1000), (3, 1000), (4, 6)])
def test_device_loop_equals_host_steps(nmg, built, sessions, case, prec, restart, maxit):
    """Restart cycles run as on-device graph loops take the same decisions and
    produce the same iterate, bit for bit, as cycles stepped by the host
    (several cycles with restart 3; the iteration limit reached mid-cycle)."""
    s, _ = built[case]
    S = sessions[case]
    b = cu(s.rhs, np.float64)
    out = []
    for graph in (1, 2):
        x = torch.empty_like(b)
        info = nmg.nmg_solve_info()
        st = nmg.nmg_solve(S.handle, b, x, _opts(nmg, precision=prec, use_graph=graph, restart=restart, maxit=maxit),
                           info)
        out.append((st, info.iterations, info.restarts, info.device_loop, x))
    (st1, it1, rs1, dl1, x1), (st2, it2, rs2, dl2, x2) = out
    assert (dl1, dl2) == (0, 1)
    assert (st1, it1, rs1) == (st2, it2, rs2)
    assert it1 <= maxit
    assert st1 == 0 or (st1 == nmg.NMG_ERR_NOT_CONVERGED and it1 == maxit)
    if maxit == 1000:
        assert st1 == 0
    assert torch.equal(x1, x2)


def _opts(nmg, **kw):
    from paper_1904_02401_gb300.session import solve_opts
    return solve_opts(**kw)


def test_solve_host_buffers_and_determinism(nmg, built, sessions):
    s, h = built["2d_24x40_3lev"]
    S = sessions["2d_24x40_3lev"]
    b = cu(s.rhs, np.float64)
    x1 = torch.empty_like(b)
    x2 = torch.empty_like(b)
    S.solve(b, x1, precision=1)
    S.solve(b, x2, precision=1)
    assert torch.equal(x1, x2)
    bh = np.ascontiguousarray(s.rhs)
    xh = np.zeros_like(bh)
    info = S.solve(bh, xh, precision=1)
    assert info.status == 0
    np.testing.assert_array_equal(xh, host(x1))


def test_error_paths(nmg, built):
    from paper_1904_02401_gb300.session import Session
    s, _ = built["2d_32x32_3lev"]
    lv = [(l.row_ptr, l.col_idx, l.vals) for l in s.levels]
    S = Session(2, s.problem.n, [], s.dirichlet, nlevels=len(lv))
    # column outside the Q1 stencil
    rp, ci, v = lv[0]
    bad = ci.copy()
    bad[5] = (bad[5] + 7) % (rp.size - 1)
    assert nmg.nmg_set_jacobian(S.handle, 0, rp.size - 1, ci.size, rp, bad, v, 0) == nmg.NMG_ERR_INVALID
    # NaN value
    vn = v.copy()
    vn[3, 0, 0] = np.nan
    assert nmg.nmg_set_jacobian(S.handle, 0, rp.size - 1, ci.size, rp, ci, vn, 0) == nmg.NMG_ERR_NONFINITE
    # singular patch: a zero matrix on level 1
    rp1, ci1, v1 = lv[1]
    assert nmg.nmg_set_jacobian(S.handle, 1, rp1.size - 1, ci1.size, rp1, ci1, np.zeros_like(v1), 0) == \
        nmg.NMG_ERR_SINGULAR_PATCH
    # solve before all levels are set
    b = cu(s.rhs, np.float64)
    x = torch.empty_like(b)
    info = nmg.nmg_solve_info()
    from paper_1904_02401_gb300.session import solve_opts
    assert nmg.nmg_solve(S.handle, b, x, solve_opts(), info) == nmg.NMG_ERR_INVALID
    for lev, (a, c, d) in enumerate(lv):
        S.set_level(lev, a, c, d)
    # maxit reached
    assert nmg.nmg_solve(S.handle, b, x, solve_opts(maxit=1), info) == nmg.NMG_ERR_NOT_CONVERGED
    assert info.iterations == 1
    # non-finite right-hand side
    bn = s.rhs.copy()
    bn[10] = np.inf
    assert nmg.nmg_solve(S.handle, cu(bn, np.float64), x, solve_opts(), info) == nmg.NMG_ERR_NONFINITE
    # unprepared precision and bad options
    assert nmg.nmg_solve(S.handle, b, x, solve_opts(restart=0), info) == nmg.NMG_ERR_INVALID
    S.close()
    S2 = Session(2, s.problem.n, lv, s.dirichlet, precisions=1 << 1)
    assert nmg.nmg_solve(S2.handle, b, x, solve_opts(precision=0), info) == nmg.NMG_ERR_INVALID
    S2.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_engines_agree(nmg, built, sessions, case, prec):
    """One-kernel-per-step (plain and graph), fused, persistent and cluster-tail
    V-cycles run the same element code in the same order: their results are
    bitwise identical.  The tails cover the two coarsest levels, and the whole
    V-cycle (finest level included, written to the caller's z)."""
    from paper_1904_02401_gb300.session import solve_opts
    s, h = built[case]
    S = sessions[case]
    dt = vdtype(prec)
    r = cu(s.rhs.astype(dt), dt)
    p1 = int(np.prod([nk // 2 ** (s.problem.levels - 2) // 2 for nk in s.problem.n]))   # patches of level 1
    outs = []
    for engine, graph, tail in ((nmg.NMG_ENGINE_KERNELS, 0, 0), (nmg.NMG_ENGINE_KERNELS, 1, 0),
                                (nmg.NMG_ENGINE_PERSISTENT, 0, 0), (nmg.NMG_ENGINE_FUSED, 0, 0),
                                (nmg.NMG_ENGINE_FUSED, 1, 0), (nmg.NMG_ENGINE_KERNELS, 0, p1),
                                (nmg.NMG_ENGINE_FUSED, 1, p1), (nmg.NMG_ENGINE_KERNELS, 1, 1 << 30),
                                (nmg.NMG_ENGINE_FUSED, 0, 1 << 30)):
        z = torch.zeros_like(r)
        o = solve_opts(precision=prec, use_graph=graph, engine=engine, tail_patches=tail)
        nmg.check(nmg.nmg_vcycle(S.handle, o, r, z))
        outs.append(z)
    # tile-fused steps: on level 1 only, on every level (finest included), above a cluster tail
    for graph, tail, tile in ((0, 0, p1), (0, 0, 1 << 30), (1, 0, 1 << 30), (1, p1, 1 << 30)):
        z = torch.zeros_like(r)
        o = solve_opts(precision=prec, use_graph=graph, engine=nmg.NMG_ENGINE_KERNELS, tail_patches=tail,
                       tile_patches=tile)
        nmg.check(nmg.nmg_vcycle(S.handle, o, r, z))
        outs.append(z)
    for k in range(1, len(outs)):
        assert torch.equal(outs[0], outs[k]), k


@pytest.mark.parametrize("case", ["2d_24x40_3lev", "3d_8x12x16_3lev"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nu", [(1, 1), (1, 3), (3, 1), (0, 2), (2, 0), (0, 0)])
@pytest.mark.parametrize("weighting", [0, 1])
def test_tile_steps_agree(nmg, built, sessions, case, prec, nu, weighting):
    """Tile-fused smoothing steps (one launch per Vanka step on a tile level,
    the pre-smoothing's last step also restricting) give the V-cycle of the
    one-kernel-per-pass path bit for bit, for any numbers of pre- and
    post-smoothing steps (the iterate's buffer parity, the zero first iterate
    and the skipped steps), both weightings of Eq. (vanka), on ragged tiles."""
    from paper_1904_02401_gb300.session import solve_opts
    s, h = built[case]
    S = sessions[case]
    dt = vdtype(prec)
    r = cu(s.rhs.astype(dt), dt)
    om = 0.8 if weighting == nmg.NMG_WEIGHT_AVERAGE else 0.3
    outs = []
    for tile in (0, 1 << 30):
        z = torch.zeros_like(r)
        o = solve_opts(precision=prec, use_graph=0, engine=nmg.NMG_ENGINE_KERNELS, nu1=nu[0], nu2=nu[1],
                       weighting=weighting, omega=om, tile_patches=tile)
        nmg.check(nmg.nmg_vcycle(S.handle, o, r, z))
        outs.append(z)
    assert torch.equal(outs[0], outs[1])
    assert torch.isfinite(outs[0]).all()


@pytest.mark.parametrize("case", list(CASES))
def test_solve_fp64_persistent_engine(nmg, built, sessions, case):
    s, h = built[case]
    S = sessions[case]
    hist = []
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8, history=hist)
    b = cu(s.rhs, np.float64)
    x = torch.empty_like(b)
    info = S.solve(b, x, precision=0, engine=nmg.NMG_ENGINE_PERSISTENT)
    assert info.status == 0
    assert _iteration_tie_ok(info.iterations, info_o["iterations"], hist, 1e-8)
    assert rel(host(x), xo) <= 1e-8
