"""Full-size workloads in the launch configuration bench.py times (CUDA graphs,
caller-owned stream).

* 2d 256x256 (7 levels) and 3d 32^3 (4 levels): the whole oracle solve runs,
  so the FP64 path is compared element by element (equal iteration counts,
  solution relative error <= 1e-8) and the mixed paths by true residual and
  forward error.
* 3d 96^3 (6 levels, 3.65M unknowns): the oracle cannot invert its 110,592
  patch matrices in the test's time, so sampled outputs are checked one by one
  (block rows of A x, patch inverses, the smoothed value at sampled nodes) and
  the solves by properties that hold at any size (true FP64 residual <= 1e-8).
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import build_system, config_problem

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _session(s, stream, precisions=0):
    from paper_1904_02401_gb300.session import Session
    return Session(s.problem.dim, s.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet,
                   precisions=precisions, stream=stream.cuda_stream)


def _true_rel_residual(level, b, x):
    import scipy.sparse as sp
    nc = level.vals.shape[1]
    A = sp.bsr_matrix((level.vals, level.col_idx, level.row_ptr), shape=(level.nodes * nc,) * 2)
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


@pytest.mark.parametrize("name", ["cfg2", "cfg3"])
def test_full_solve_against_oracle(name):
    _need_gpu()
    from oracle.fgmres import fgmres
    from oracle.multigrid import Hierarchy
    s = build_system(config_problem(name))
    h = Hierarchy(s.levels, s.dirichlet)
    hist = []
    xo, info_o = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8, history=hist)
    stream = torch.cuda.Stream()
    S = _session(s, stream)
    try:
        b = torch.from_numpy(s.rhs).cuda()
        x = torch.empty_like(b)
        with torch.cuda.stream(stream):
            info = S.solve(b, x, precision=0, use_graph=1)
        assert info.status == 0
        near = any(1e-8 / 1.01 <= v <= 1e-8 * 1.01 for v in hist[-2:])
        assert info.iterations == info_o["iterations"] or (near and abs(info.iterations - info_o["iterations"]) <= 1)
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
        for prec in (1, 2):
            with torch.cuda.stream(stream):
                info = S.solve(b, x, precision=prec, use_graph=1)
            assert info.status == 0
            xg = x.cpu().numpy()
            assert _true_rel_residual(s.fine, s.rhs, xg) <= 1e-8
            assert info.iterations <= info_o["iterations"] + 3
    finally:
        S.close()


@pytest.fixture(scope="module")
def big():
    _need_gpu()
    s = build_system(config_problem("cfg4"))
    stream = torch.cuda.Stream()
    S = _session(s, stream)
    yield s, S, stream
    S.close()


def _row_products(level, x, rows):
    nc = level.vals.shape[1]
    out = np.zeros((rows.size, nc))
    for k, i in enumerate(rows):
        lo, hi = level.row_ptr[i], level.row_ptr[i + 1]
        cols = level.col_idx[lo:hi]
        out[k] = np.einsum("brc,bc->r", level.vals[lo:hi], x.reshape(-1, nc)[cols])
    return out


def _sample_nodes(level, rng, k=1500):
    n = level.nodes
    return np.unique(np.concatenate([rng.integers(0, n, k), [0, 1, n - 2, n - 1, n // 2]]))


def test_96cube_matvec_sampled_rows(big):
    from paper_1904_02401_gb300 import nmg
    s, S, stream = big
    L = len(s.levels) - 1
    rng = np.random.default_rng(1)
    rows = _sample_nodes(s.fine, rng)
    nc = 4
    x = rng.standard_normal(s.unknowns)
    ref = _row_products(s.fine, x, rows)
    scale = _row_products(type(s.fine)(s.fine.cells, s.fine.row_ptr, s.fine.col_idx, np.abs(s.fine.vals)),
                          np.abs(x), rows) + 1e-300
    for prec, dt, tol in ((0, torch.float64, 1e-13), (1, torch.float32, 1e-5)):
        xd = torch.from_numpy(x).to(dt).cuda()
        y = torch.empty_like(xd)
        with torch.cuda.stream(stream):
            nmg.check(nmg.nmg_matvec(S.handle, L, prec, xd, y))
        yg = y.double().cpu().numpy().reshape(-1, nc)[rows]
        if prec == 1:
            xr = xd.double().cpu().numpy()
            vals32 = s.fine.vals.astype(np.float32).astype(np.float64)
            ref = _row_products(type(s.fine)(s.fine.cells, s.fine.row_ptr, s.fine.col_idx, vals32), xr, rows)
        assert np.max(np.abs(yg - ref) / scale) < tol


def test_96cube_patch_inverses_and_smoothing_sampled(big):
    from oracle.bsr import BlockMatrix
    from oracle.mesh import node_coords, patch_nodes
    from paper_1904_02401_gb300 import nmg
    s, S, stream = big
    L = len(s.levels) - 1
    fine = s.fine
    A = BlockMatrix(fine.row_ptr, fine.col_idx, fine.vals)
    pn = patch_nodes(fine.cells)                      # (110592, 27)
    rng = np.random.default_rng(2)
    sel = np.unique(np.concatenate([rng.integers(0, pn.shape[0], 40), [0, pn.shape[0] - 1]]))
    nc = 4
    n_p = 108

    def patch_matrix(p):
        nodes = pn[p]
        blk = A.block_lookup(nodes[:, None], nodes[None, :])
        return blk.transpose(0, 2, 1, 3).reshape(n_p, n_p)

    for p in sel:
        Ap = patch_matrix(p)
        ref = np.linalg.inv(Ap)
        out = np.empty((1, n_p, n_p))
        nmg.check(nmg.nmg_get_patch_inverses(S.handle, L, 0, int(p), 1, out))
        assert np.abs(out[0] - ref).max() <= 1e-7 * np.abs(ref).max()
    # one smoothing step from zero at sampled nodes: x_i = omega/m_i sum_{P ni i} (A_P^{-1} b_P)_i
    b = s.rhs
    bd = torch.from_numpy(b).cuda()
    x = torch.empty_like(bd)
    with torch.cuda.stream(stream):
        nmg.check(nmg.nmg_smooth(S.handle, L, 0, bd, x, 1, 1, 0.8, nmg.NMG_WEIGHT_AVERAGE))
    xg = x.cpu().numpy().reshape(-1, nc)
    node_patches = {}
    for node in _sample_nodes(fine, rng, 60):
        node_patches[int(node)] = np.nonzero((pn == node).any(axis=1))[0]
    for node, plist in node_patches.items():
        acc = np.zeros(nc)
        for p in plist:
            loc = int(np.nonzero(pn[p] == node)[0][0])
            dofs = (pn[p][:, None] * nc + np.arange(nc)).reshape(-1)
            c = np.linalg.solve(patch_matrix(p), b[dofs])
            acc += c[loc * nc:(loc + 1) * nc]
        ref = 0.8 * acc / len(plist)
        assert np.allclose(xg[node], ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max() + 1e-300)


@pytest.mark.parametrize("prec", [1, 0, 2])
def test_96cube_solve_residual(big, prec):
    s, S, stream = big
    b = torch.from_numpy(s.rhs).cuda()
    x = torch.empty_like(b)
    with torch.cuda.stream(stream):
        info = S.solve(b, x, precision=prec, use_graph=1)
    assert info.status == 0, info.status
    assert _true_rel_residual(s.fine, s.rhs, x.cpu().numpy()) <= 1e-8
    assert abs(info.rel_residual - _true_rel_residual(s.fine, s.rhs, x.cpu().numpy())) < 1e-10
    assert info.iterations <= 60


@pytest.mark.parametrize("prec", [1, 2])
def test_96cube_multi_vector(big, prec):
    """8 columns through the multi-vector V-cycle (graph replay, as bench.py's
    multi_rhs times it) equal single V-cycles bit for bit at full size, and a
    2-column multi-vector solve equals the single solves (counts, iterates)
    and meets the true FP64 residual."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    s, S, stream = big
    rng = np.random.default_rng(77)
    mask = s.dirichlet.astype(bool)
    cols = [s.rhs]
    for _ in range(7):
        v = rng.uniform(-1.0, 1.0, s.rhs.size)
        v[mask] = 0.0
        cols.append(v)
    B = torch.from_numpy(np.stack(cols)).cuda()
    R = B.to(torch.float32)
    Z = torch.full_like(R, float("nan"))
    with torch.cuda.stream(stream):
        nmg.check(nmg.nmg_vcycle_many(S.handle, solve_opts(precision=prec, use_graph=1), 8, R, Z))
        for k in (0, 3, 7):
            z = torch.zeros_like(R[k])
            nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=0, engine=nmg.NMG_ENGINE_KERNELS),
                                     R[k].contiguous(), z))
            torch.cuda.synchronize()
            assert torch.equal(Z[k], z), k
        X = torch.zeros_like(B[:2])
        infos = S.solve_many(B[:2].contiguous(), X, 2, precision=prec)
        for k in range(2):
            x = torch.empty_like(B[k])
            info = S.solve(B[k].contiguous(), x, precision=prec, use_graph=0, engine=nmg.NMG_ENGINE_KERNELS)
            assert infos[k].status == info.status == 0
            assert infos[k].iterations == info.iterations
            assert torch.equal(X[k], x)
            assert _true_rel_residual(s.fine, cols[k], X[k].cpu().numpy()) <= 1e-8


# ----------------------------------------------------------------------------
# FP32 / BF16 paths at 96^3 node by node: every CTA of the streaming Vanka
# apply walks many more chunks than its ring has stages (tests/rounding_bounds.py
# states the tolerances)
# ----------------------------------------------------------------------------

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "vcycle_96cube_oracle.txt")


def _golden_vcycle():
    """The FP64 oracle's V(2,2) cycle of the workload's right-hand side at
    sampled nodes (tests/golden/make_vcycle_96cube.py), with its largest entry
    and, per component, how far the binary32 model of the cycle lies from it."""
    head = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("# max_abs"):
                key, *vals = line[2:].split()
                head[key] = np.array([float(v) for v in vals])
    data = np.loadtxt(GOLDEN)
    return data[:, 0].astype(np.int64), data[:, 1:], head


@pytest.mark.parametrize("prec", [1, 2])
def test_96cube_one_vanka_step_sampled(big, prec):
    """One FP32/BF16 Vanka step from a random iterate at sampled nodes, each
    entry within its first-order rounding bound."""
    from oracle.bsr import BlockMatrix
    from oracle.mesh import patch_nodes
    from paper_1904_02401_gb300 import nmg
    from rounding_bounds import to_storage32, vanka_step_and_bound
    s, S, stream = big
    L = len(s.levels) - 1
    fine = s.fine
    nc, dim = 4, 3
    A = BlockMatrix(fine.row_ptr, fine.col_idx, fine.vals)
    pn = patch_nodes(fine.cells)
    rng = np.random.default_rng(12 + prec)
    b = to_storage32(rng.uniform(-1, 1, s.unknowns))
    x0 = to_storage32(rng.uniform(-1, 1, s.unknowns))
    targets = _sample_nodes(fine, rng, 80)
    plist = {int(t): np.nonzero((pn == t).any(axis=1))[0] for t in targets}
    patches = np.unique(np.concatenate(list(plist.values())))
    pnodes = np.unique(pn[patches])
    d = np.zeros(s.unknowns)
    abs_ax = np.zeros(s.unknowns)
    absA = type(fine)(fine.cells, fine.row_ptr, fine.col_idx, np.abs(fine.vals))
    rows = (pnodes[:, None] * nc + np.arange(nc)).reshape(-1)
    d[rows] = b[rows] - _row_products(fine, x0, pnodes).reshape(-1)
    abs_ax[rows] = _row_products(absA, np.abs(x0), pnodes).reshape(-1)
    nodes = pn[patches]
    Ap = A.block_lookup(nodes[:, :, None], nodes[:, None, :]).transpose(0, 1, 3, 2, 4).reshape(
        patches.size, 27 * nc, 27 * nc)
    inv = np.linalg.inv(Ap)
    dofs = (nodes[:, :, None] * nc + np.arange(nc)).reshape(patches.size, -1)
    w = np.ones(s.unknowns)
    for t, pl in plist.items():
        w[t * nc:(t + 1) * nc] = 1.0 / len(pl)
    ref, bound = vanka_step_and_bound(inv, dofs, b, x0, d, abs_ax, w, 0.8, prec, dim, nc)
    xd = torch.from_numpy(x0.astype(np.float32)).cuda()
    with torch.cuda.stream(stream):
        nmg.check(nmg.nmg_smooth(S.handle, L, prec, torch.from_numpy(b.astype(np.float32)).cuda(), xd, 1, 0, 0.8,
                                 nmg.NMG_WEIGHT_AVERAGE))
    stream.synchronize()
    got = xd.double().cpu().numpy()
    sel = (np.array(sorted(plist))[:, None] * nc + np.arange(nc)).reshape(-1)
    err = np.abs(got[sel] - ref[sel])
    assert np.all(err <= bound[sel]), (err / bound[sel]).max()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("many", [False, True])
def test_96cube_vcycle_sampled_against_oracle(big, prec, many):
    """The FP32/BF16 V(2,2) cycle of the workload's right-hand side (graph
    replay, as the solve runs it), and column 0 and 5 of an 8-column
    multi-vector cycle, against the FP64 oracle's cycle at 1,114 sampled
    nodes."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    from rounding_bounds import vcycle_tolerance, within
    s, S, stream = big
    nodes, zref, head = _golden_vcycle()
    nc = 4
    tol = vcycle_tolerance(head["max_abs_dz_%s_model" % {1: "fp32", 2: "bf16"}[prec]], head["max_abs_z"][0], nc)
    r = torch.from_numpy(s.rhs.astype(np.float32)).cuda()
    outs = []
    with torch.cuda.stream(stream):
        if many:
            rng = np.random.default_rng(8)
            mask = s.dirichlet.astype(bool)
            cols = []
            for k in range(8):
                v = s.rhs.astype(np.float32) if k in (0, 5) else rng.uniform(-1, 1, s.unknowns).astype(np.float32)
                v[mask] = 0.0
                cols.append(v)
            R = torch.from_numpy(np.stack(cols)).cuda()
            Z = torch.full_like(R, float("nan"))
            nmg.check(nmg.nmg_vcycle_many(S.handle, solve_opts(precision=prec, use_graph=1), 8, R, Z))
            outs = [Z[0], Z[5]]
        else:
            z = torch.zeros_like(r)
            nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=1), r, z))
            outs = [z]
    stream.synchronize()
    for z in outs:
        got = z.double().cpu().numpy().reshape(-1, nc)[nodes]
        err = got - zref
        assert within(err, tol, nc).all(), (np.abs(err).max(axis=0), tol)
