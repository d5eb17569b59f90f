"""Element-wise parity of the FP32 and BF16 paths with the FP64 oracle at full
workload size: 2d 256x256 (7 levels, 16,384 finest patches of 27 unknowns) and
3d 32^3 (4 levels, 4,096 finest patches of 108 unknowns).  At these sizes every
CTA of the streaming Vanka apply walks more chunks of inverses than its ring
has stages, so the ring wraps and the barrier phases flip; the launch
configuration is the one bench.py times (caller-owned stream, graphs).

Tolerances (tests/rounding_bounds.py):
* one Vanka step (Eq. (vanka)): every entry within its first-order rounding
  bound B (FP32 arithmetic, one rounding of the stored inverses);
* two steps and whole V(2,2) cycles: every entry within 8 times the largest
  deviation (in its component) of the oracle run the binary32 way (binary32
  matrices, vectors and arithmetic, inverses rounded to the storage format),
  plus 16 u max|z|;
* solves: the true FP64 residual <= 1e-8, and the forward error against a
  tightly converged FP64 oracle solve within max(1e-7, 20x the FP64 oracle's
  own forward error at rtol 1e-8).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import build_system, config_problem
from oracle.fgmres import fgmres
from oracle.multigrid import Hierarchy
from oracle.precision import with_fp32_arithmetic
from oracle.vanka import overlap_weights, vanka_step
from rounding_bounds import model_vcycle_dz, to_storage32, vanka_step_and_bound, vcycle_tolerance, within

pytestmark = pytest.mark.gpu

STORE = {1: "fp32", 2: "bf16"}


@pytest.fixture(scope="module", params=["cfg2", "cfg3"])
def full(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300.session import Session
    s = build_system(config_problem(request.param))
    h = Hierarchy(s.levels, s.dirichlet)
    stream = torch.cuda.Stream()
    S = Session(s.problem.dim, s.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet,
                stream=stream.cuda_stream)
    yield request.param, s, h, S, stream
    S.close()


def _f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("weighting", [0, 1])
@pytest.mark.parametrize("x_zero", [1, 0])
def test_one_vanka_step_every_entry(full, prec, weighting, x_zero):
    from paper_1904_02401_gb300 import nmg
    name, s, h, S, stream = full
    lev = len(h.levels) - 1
    L = h.levels[lev]
    dim, nc = s.problem.dim, s.problem.ncomp
    omega = 0.8 if weighting == 0 else 0.3
    rng = np.random.default_rng(31 + prec + 2 * weighting)
    b = to_storage32(rng.uniform(-1, 1, L.A.size))
    x0 = np.zeros(L.A.size) if x_zero else to_storage32(rng.uniform(-1, 1, L.A.size))
    d = b - L.A.matvec(x0)
    abs_ax = abs(L.A.csr) @ np.abs(x0)
    w = overlap_weights(L.dofs, L.A.size, "average" if weighting == 0 else "sum")
    ref, bound = vanka_step_and_bound(L.Ainv, L.dofs, b, x0, d, abs_ax, w, omega, prec, dim, nc)
    np.testing.assert_allclose(ref, vanka_step(L.A, L.Ainv, L.dofs, b, x0, omega, w), rtol=1e-12, atol=1e-14)
    xd = _f32(x0 if not x_zero else rng.uniform(-1, 1, L.A.size))    # x_is_zero ignores the contents
    with torch.cuda.stream(stream):
        nmg.check(nmg.nmg_smooth(S.handle, lev, prec, _f32(b), xd, 1, x_zero, omega, weighting))
    stream.synchronize()
    got = xd.double().cpu().numpy()
    err = np.abs(got - ref)
    worst = int(np.argmax(err / (bound + 1e-300)))
    assert np.all(err <= bound), (name, worst, err[worst], bound[worst])


@pytest.mark.parametrize("prec", [1, 2])
def test_two_vanka_steps_every_entry(full, prec):
    from paper_1904_02401_gb300 import nmg
    name, s, h, S, stream = full
    lev = len(h.levels) - 1
    L = h.levels[lev]
    rng = np.random.default_rng(41 + prec)
    b = to_storage32(rng.uniform(-1, 1, L.A.size))
    x0 = to_storage32(rng.uniform(-1, 1, L.A.size))
    ref = vanka_step(L.A, L.Ainv, L.dofs, b, vanka_step(L.A, L.Ainv, L.dofs, b, x0, 0.8, L.weight), 0.8, L.weight)
    Lm = with_fp32_arithmetic(h, STORE[prec]).levels[lev]
    b32, om32 = b.astype(np.float32), np.float32(0.8)
    rs = vanka_step(Lm.A, Lm.Ainv, L.dofs, b32, vanka_step(Lm.A, Lm.Ainv, L.dofs, b32, x0.astype(np.float32), om32,
                                                          Lm.weight), om32, Lm.weight)
    nc = s.problem.ncomp
    tol = vcycle_tolerance(np.abs(rs - ref).reshape(-1, nc).max(axis=0), np.abs(ref).max(), nc)
    xd = _f32(x0)
    with torch.cuda.stream(stream):
        nmg.check(nmg.nmg_smooth(S.handle, lev, prec, _f32(b), xd, 2, 0, 0.8, nmg.NMG_WEIGHT_AVERAGE))
    stream.synchronize()
    err = xd.double().cpu().numpy() - ref
    assert within(err, tol, nc).all(), (name, np.abs(err).reshape(-1, nc).max(axis=0), tol)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_vcycle_every_entry(full, prec, use_graph):
    """z = V(2,2) r for the workload's right-hand side, engine as the solve uses
    it (autotuned), plain launches and graph replay."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    name, s, h, S, stream = full
    r = to_storage32(s.rhs)
    nc = s.problem.ncomp
    dz, ref = model_vcycle_dz(h, r, STORE[prec], nc)
    tol = vcycle_tolerance(dz, np.abs(ref).max(), nc)
    z = torch.zeros(r.size, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=use_graph), _f32(r), z))
    stream.synchronize()
    err = z.double().cpu().numpy() - ref
    assert within(err, tol, nc).all(), (name, np.abs(err).reshape(-1, nc).max(axis=0), tol)


@pytest.mark.parametrize("prec", [1, 2])
def test_engines_agree_at_full_size(full, prec):
    """At this size the streaming apply runs its wrapping ring and, on the 2d
    levels of at least 4096 patches, two patches a warp; the per-step kernels
    (plain and replayed as a graph) and the persistent engine (its own
    double-buffered apply) sum the same terms in the same order, so their
    V-cycles agree bit for bit."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    name, s, h, S, stream = full
    r = _f32(to_storage32(s.rhs))
    outs = []
    for engine, graph in ((nmg.NMG_ENGINE_KERNELS, 0), (nmg.NMG_ENGINE_KERNELS, 1), (nmg.NMG_ENGINE_PERSISTENT, 0)):
        z = torch.zeros_like(r)
        with torch.cuda.stream(stream):
            nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=graph, engine=engine), r, z))
        stream.synchronize()
        outs.append(z)
    assert torch.isfinite(outs[0]).all()
    for k in range(1, len(outs)):
        assert torch.equal(outs[0], outs[k]), k


@pytest.mark.parametrize("prec", [1, 2])
def test_vcycle_many_columns_every_entry(full, prec):
    """Columns 0 and 5 of an 8-column multi-vector V-cycle against the oracle."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    name, s, h, S, stream = full
    r = to_storage32(s.rhs)
    nc = s.problem.ncomp
    dz, ref = model_vcycle_dz(h, r, STORE[prec], nc)
    tol = vcycle_tolerance(dz, np.abs(ref).max(), nc)
    rng = np.random.default_rng(5)
    cols = np.stack([r if k in (0, 5) else to_storage32(rng.uniform(-1, 1, r.size)) * (1 - s.dirichlet)
                     for k in range(8)])
    R = _f32(cols)
    Z = torch.full_like(R, float("nan"))
    with torch.cuda.stream(stream):
        nmg.check(nmg.nmg_vcycle_many(S.handle, solve_opts(precision=prec, use_graph=1), 8, R, Z))
    stream.synchronize()
    for k in (0, 5):
        err = Z[k].double().cpu().numpy() - ref
        assert within(err, tol, nc).all(), (name, k, np.abs(err).reshape(-1, nc).max(axis=0), tol)


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_solve_forward_error(full, prec):
    """The mixed-precision solve (FP64 FGMRES, reduced-precision V-cycle) reaches
    the FP64 true residual 1e-8 and lies as close to the exact solution as the
    FP64 oracle's own solve at the same rtol (within max(1e-7, 20x))."""
    name, s, h, S, stream = full
    xt, _ = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-12)
    xo, _ = fgmres(h.fine.A.matvec, h.vcycle, s.rhs, rtol=1e-8)
    b = torch.from_numpy(s.rhs).cuda()
    x = torch.empty_like(b)
    with torch.cuda.stream(stream):
        info = S.solve(b, x, precision=prec, use_graph=2)
    assert info.status == 0
    xg = x.cpu().numpy()
    relres = np.linalg.norm(s.rhs - h.fine.A.matvec(xg)) / np.linalg.norm(s.rhs)
    assert relres <= 1e-8
    err = np.linalg.norm(xg - xt) / np.linalg.norm(xt)
    err_o = np.linalg.norm(xo - xt) / np.linalg.norm(xt)
    err_vs_oracle = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print(f"{name} prec {prec}: forward error {err:.2e} (FP64 oracle {err_o:.2e}), vs oracle solve {err_vs_oracle:.2e}")
    assert err <= max(1e-7, 20 * err_o), (err, err_o)
