"""The integer float -> double widening used by the FP64 operator product
(elem.cuh widen_exact) restated bit for bit in Python and checked against
numpy's conversion on every class of binary32 value: zeros, subnormals (all
23 leading-one positions), normals across the exponent range, infinities.
The device code is this mapping; the GPU solves exercise it in place."""

import numpy as np


def widen_exact(f32):
    u = int(np.float32(f32).view(np.uint32))
    sign = (u & 0x80000000) << 32
    e = (u >> 23) & 0xFF
    m = u & 0x7FFFFF
    if 1 <= e <= 254:
        bits = sign | ((e + 896) << 52) | (m << 29)
    elif e == 0xFF:
        bits = sign | (0x7FF << 52) | (m << 29)
    elif m == 0:
        bits = sign
    else:
        clz = 32 - m.bit_length()
        sh = clz - 8
        m = (m << sh) & 0x7FFFFF
        bits = sign | ((897 - sh) << 52) | (m << 29)
    return np.array([bits], dtype=np.uint64).view(np.float64)[0]


def _values():
    rng = np.random.default_rng(5)
    vals = [0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, np.finfo(np.float32).max, np.finfo(np.float32).tiny]
    # one subnormal per leading-one position, plus random fractions
    for p in range(23):
        vals.append(np.uint32(1 << p).view(np.float32))
        vals.append(np.uint32((1 << p) | int(rng.integers(0, 1 << p + 1)) & ((1 << (p + 1)) - 1)).view(np.float32))
    vals += list(rng.standard_normal(2000).astype(np.float32) * np.float32(10.0) ** rng.integers(-30, 30, 2000))
    return np.array(vals, dtype=np.float32)


def test_widen_matches_conversion():
    for f in _values():
        got = widen_exact(f)
        want = np.float64(f)
        assert np.array([got]).view(np.uint64)[0] == np.array([want]).view(np.uint64)[0], (f, got, want)


def test_widen_nan_stays_nan():
    assert np.isnan(widen_exact(np.float32(np.nan)))
