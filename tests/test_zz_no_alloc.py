"""nmg_vanka_correct_noalloc: the Vanka correction for callers that cannot allocate.

Callers that own all device memory in a fixed arena, or whose hot loop may not
call cudaMalloc, use this entry point: it takes every input and output from
the caller and keeps its scratch in a fixed device array of the library.  The
test checks, on two calls in a row in 2d and 3d with both combinations of the
overlapping corrections, that it gives what the regular smoothing call
(nmg_smooth, which uses the hierarchy's own scratch) gives, that its first step
matches the FP64 oracle's, and that a mesh too large for the fixed array is
refused.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _inverses_in_library_layout(nmg, handle, level, prec, patches, n_p):
    """Patch inverses read back through the C ABI, laid out as the library stores them."""
    rowmajor = np.empty((patches, n_p, n_p))
    nmg.check(nmg.nmg_get_patch_inverses(handle, level, prec, 0, patches, rowmajor))
    esize = {0: 8, 1: 4, 2: 2}[prec]
    per = 16 // esize
    stride = (n_p * n_p + per - 1) // per * per
    buf = np.zeros((patches, stride))
    buf[:, : n_p * n_p] = rowmajor.transpose(0, 2, 1).reshape(patches, -1)   # column-major per patch
    dtype = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[prec]
    return torch.from_numpy(buf.reshape(-1)).to(dtype).cuda(), stride


MESHES = {
    2: dict(dim=2, n=(32, 24), levels=3, solid=(0, +1, 0.6)),
    3: dict(dim=3, n=(8, 8, 8), levels=2, solid=(2, -1, 0.25)),
}


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("weighting", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_vanka_matches_regular_smoothing(dim, weighting, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gen import Problem, build_system
    from oracle.multigrid import Hierarchy
    from oracle.vanka import overlap_weights, vanka_step
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import Session
    from rounding_bounds import to_storage32, vanka_step_and_bound

    p = Problem(**MESHES[dim])
    s = build_system(p)
    cells = s.fine.cells
    level = len(s.levels) - 1
    n_p = 3 ** dim * (dim + 1)
    patches = int(np.prod([c // 2 for c in cells]))
    n = s.unknowns
    omega = 0.8 if weighting == 0 else 0.3
    vdt = torch.float64 if prec == 0 else torch.float32
    tol = 1e-12 if prec == 0 else 1e-5
    rng = np.random.default_rng(21)
    with Session(dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet) as S:
        inv, stride = _inverses_in_library_layout(nmg, S.handle, level, prec, patches, n_p)
        b = torch.from_numpy(rng.standard_normal(n)).to(vdt).cuda()
        x0 = torch.from_numpy(rng.standard_normal(n)).to(vdt).cuda()

        # call 1: zero initial guess, defect = b
        x_ref = x0.clone()
        nmg.check(nmg.nmg_smooth(S.handle, level, prec, b, x_ref, 1, 1, omega, weighting))
        x_new = x0.clone()
        nmg.check(nmg.nmg_vanka_correct_noalloc(dim, cells, prec, inv, stride, b, x_new, omega, weighting, 1, None))
        torch.cuda.synchronize()
        err1 = (x_new - x_ref).abs().max().item() / x_ref.abs().max().item()
        assert err1 <= tol, err1
        # ... and against the FP64 oracle's step (FP32 / BF16: every entry within its rounding bound)
        h = Hierarchy(s.levels, s.dirichlet)
        L = h.fine
        bh = b.double().cpu().numpy()
        w = overlap_weights(L.dofs, n, "average" if weighting == 0 else "sum")
        got = x_new.double().cpu().numpy()
        if prec == 0:
            ref = vanka_step(L.A, L.Ainv, L.dofs, bh, np.zeros(n), omega, w)
            assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max()
        else:
            zero = np.zeros(n)
            ref, bound = vanka_step_and_bound(L.Ainv, L.dofs, to_storage32(bh), zero, bh, zero, w, omega, prec,
                                              dim, dim + 1)
            assert np.all(np.abs(got - ref) <= bound)

        # call 2: continue from the result, defect d = b - A x from the regular residual call
        x_ref2 = x_ref.clone()
        nmg.check(nmg.nmg_smooth(S.handle, level, prec, b, x_ref2, 1, 0, omega, weighting))
        d = torch.empty_like(x_new)
        nmg.check(nmg.nmg_residual(S.handle, level, prec, b, x_new, d))
        x_new2 = x_new.clone()
        nmg.check(nmg.nmg_vanka_correct_noalloc(dim, cells, prec, inv, stride, d, x_new2, omega, weighting, 0, None))
        torch.cuda.synchronize()
        err2 = (x_new2 - x_ref2).abs().max().item() / x_ref2.abs().max().item()
        assert err2 <= tol, err2


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300 import nmg
    dummy = torch.zeros(16, device="cuda")
    # 3d 96^3 in FP32: 110592 patches * 108 * 4 bytes = 47.8 MB > 16 MiB
    st = nmg.nmg_vanka_correct_noalloc(3, (96, 96, 96), nmg.NMG_PREC_FP32, dummy, 108 * 108, dummy, dummy, 0.8,
                                       nmg.NMG_WEIGHT_AVERAGE, 1, None)
    assert st == nmg.NMG_ERR_INVALID
    assert "too large" in nmg.nmg_last_error()
