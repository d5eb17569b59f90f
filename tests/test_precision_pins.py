"""Pins of the oracle's storage rounding (oracle/precision.py) to the formats'
definitions: IEEE 754 binary32 and bfloat16 (the upper half of binary32), both
rounded to nearest with ties to even."""

import numpy as np
import pytest

from oracle.precision import round_bf16, round_fp32, with_stored_inverses


def test_bf16_matches_library_conversion_on_binary32_inputs():
    """On values that are exact binary32 numbers, the single-step rounding equals
    torch's float32 -> bfloat16 conversion (round to nearest even)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-40, 40, 100000))).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(round_bf16(x), ref)


def test_bf16_ties_and_spacing():
    u = 2.0 ** -8                     # unit roundoff; spacing at 1 is 2^-7
    cases = {
        1.0 + u: 1.0,                 # tie between 1 and 1 + 2^-7: even (1)
        1.0 + 3 * u: 1.0 + 2 * 2 * u,  # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
        1.0 + u + 2.0 ** -30: 1.0 + 2 * u,   # just above the tie: up (one-step rounding)
        -(1.0 + u + 2.0 ** -30): -(1.0 + 2 * u),
        3.0 * 2.0 ** -133: 3.0 * 2.0 ** -133,  # subnormal bfloat16, exact
        3.0 * 2.0 ** -140: 0.0,       # below half the smallest subnormal, 2^-133
        1.3 * 2.0 ** -130: 10.0 * 2.0 ** -133,  # subnormal spacing 2^-133
        0.0: 0.0,
    }
    for v, ref in cases.items():
        assert round_bf16(np.array([v]))[0] == ref, v
    # every value within half a spacing of its rounding
    rng = np.random.default_rng(1)
    x = rng.standard_normal(10000) * 10.0 ** rng.uniform(-10, 10, 10000)
    r = round_bf16(x)
    assert np.all(np.abs(r - x) <= u * np.abs(x))


def test_fp32_rounding():
    u = 2.0 ** -24
    assert round_fp32(np.array([1.0 + u]))[0] == 1.0
    assert round_fp32(np.array([1.0 + 3 * u]))[0] == 1.0 + 4 * u
    rng = np.random.default_rng(2)
    x = rng.standard_normal(10000) * 10.0 ** rng.uniform(-10, 10, 10000)
    assert np.all(np.abs(round_fp32(x) - x) <= u * np.abs(x))


def test_stored_inverses_copy_leaves_the_hierarchy_alone():
    from gen import Problem, build_system
    from oracle.multigrid import Hierarchy
    s = build_system(Problem(dim=2, n=(8, 8), levels=2, solid=(0, +1, 0.6)))
    h = Hierarchy(s.levels, s.dirichlet)
    inv = h.fine.Ainv.copy()
    hb = with_stored_inverses(h, "bf16")
    assert np.array_equal(h.fine.Ainv, inv)
    assert np.array_equal(hb.fine.Ainv, round_bf16(inv))
    assert hb.fine.A is h.fine.A
    z, zb = h.vcycle(s.rhs), hb.vcycle(s.rhs)
    assert 0 < np.abs(zb - z).max() <= 1e-2 * np.abs(z).max()


def test_fp32_model_runs_in_binary32_and_stays_near_the_oracle():
    """The binary32 model of the V-cycle computes in float32 and lies within a
    few thousand binary32 roundings of the FP64 cycle (FP32 inverses), and
    within the bfloat16 rounding scale with BF16 inverses; the FP64 hierarchy
    it was copied from is untouched."""
    from gen import Problem, build_system
    from oracle.multigrid import Hierarchy
    from oracle.precision import with_fp32_arithmetic
    s = build_system(Problem(dim=2, n=(16, 16), levels=3, solid=(0, +1, 0.6)))
    h = Hierarchy(s.levels, s.dirichlet)
    r = s.rhs.astype(np.float32)
    z = h.vcycle(r.astype(np.float64))
    inv = h.fine.Ainv.copy()
    z32 = with_fp32_arithmetic(h, "fp32").vcycle(r)
    zbf = with_fp32_arithmetic(h, "bf16").vcycle(r)
    assert z32.dtype == np.float32 and zbf.dtype == np.float32
    assert np.array_equal(h.fine.Ainv, inv) and h.vcycle(r.astype(np.float64)).dtype == np.float64
    m = np.abs(z).max()
    assert 0 < np.abs(z32 - z).max() <= 1e3 * 2.0 ** -24 * m
    assert np.abs(z32 - z).max() < np.abs(zbf - z).max() <= 2.0 ** -8 * m
