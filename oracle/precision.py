"""Storage rounding of the reduced-precision V-cycle (oracle side; test infrastructure).

The mixed-precision solves keep the outer FGMRES in FP64 and store the patch
inverses of Eq. (vanka) in FP32 or BF16.  Storing an inverse rounds each entry
once to the nearest value of the storage format, ties to even:

* binary32 (IEEE 754): 24 significant bits, unit roundoff 2^-24;
* bfloat16: the upper 16 bits of binary32 (8 significant bits, same exponent
  range), unit roundoff 2^-8.

The tests use these roundings to state how far a reduced-precision result may
lie from the FP64 oracle: the oracle's V-cycle run on the rounded inverses
shows the effect of one rounding of every stored inverse entry.
"""

from __future__ import annotations

import copy

import numpy as np

UNIT_ROUNDOFF = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -8}


def round_fp32(a) -> np.ndarray:
    """Nearest binary32 value of each entry (ties to even), returned as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(a) -> np.ndarray:
    """Nearest bfloat16 value of each finite entry (ties to even), as float64.

    Rounded in one step from the float64 value: with a = m 2^e, 1/2 <= |m| < 1,
    the bfloat16 neighbours of a normal number are the multiples of 2^(e-8),
    so a rounds to rint(m 2^8) 2^(e-8) (rint rounds half to even; the power-of-
    two scalings are exact).  Below the smallest normal bfloat16, 2^-126, the
    spacing is the fixed 2^-133.  Values beyond the bfloat16 range do not occur
    among patch inverses and are not handled.
    """
    x = np.asarray(a, dtype=np.float64)
    out = np.empty_like(x)
    xf, of = x.reshape(-1), out.reshape(-1)
    step = 1 << 22                       # bounded temporaries for multi-GB inverse arrays
    for lo in range(0, xf.size, step):
        c = xf[lo:lo + step]
        m, e = np.frexp(c)
        normal = np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)
        sub = np.ldexp(np.rint(np.ldexp(c, 133)), -133)
        of[lo:lo + step] = np.where(np.abs(c) < 2.0 ** -126, sub, normal)
    return out


def round_storage(a, fmt: str) -> np.ndarray:
    if fmt == "fp32":
        return round_fp32(a)
    if fmt == "bf16":
        return round_bf16(a)
    raise ValueError(fmt)


def with_stored_inverses(hierarchy, fmt: str):
    """A copy of an oracle Hierarchy whose patch inverses are rounded to the
    storage format fmt ("fp32" or "bf16"); everything else is shared and the
    arithmetic stays FP64."""
    h = copy.copy(hierarchy)
    h.levels = []
    for L in hierarchy.levels:
        c = copy.copy(L)
        if L.Ainv is not None:
            c.Ainv = round_storage(L.Ainv, fmt)
        if getattr(L, "groups", None) is not None:
            c.groups = [(dofs, round_storage(inv, fmt)) for dofs, inv in L.groups]
        h.levels.append(c)
    return h


class _Float32Matrix:
    """A level matrix rounded to binary32 whose products run in binary32."""

    def __init__(self, A):
        self.csr = A.csr.astype(np.float32)
        self.ncomp = A.ncomp
        self.nodes = A.nodes

    @property
    def size(self) -> int:
        return self.nodes * self.ncomp

    def matvec(self, x):
        return self.csr @ x


def with_fp32_arithmetic(hierarchy, fmt: str):
    """A copy of an oracle Hierarchy that runs the V-cycle the way the
    reduced-precision path does: level matrices, transfers, overlap weights and
    every vector in binary32 (NumPy float32 arithmetic), patch inverses rounded
    to the storage format fmt ("fp32" or "bf16") and held as binary32, and the
    coarsest level solved exactly in FP64 with the result rounded to binary32.
    Call its vcycle with a float32 vector.  The tests use how far this copy's
    result lies from the FP64 oracle's as the scale of the rounding errors of
    the reduced-precision V-cycle (summation orders differ from any GPU
    kernel's, so it is a model of their size, not of their values)."""
    import scipy.linalg as sla
    h = copy.copy(hierarchy)
    h.levels = []
    for L in hierarchy.levels:
        c = copy.copy(L)
        c.A = _Float32Matrix(L.A)
        if L.Ainv is not None:
            c.Ainv = round_storage(L.Ainv, fmt).astype(np.float32)
        if getattr(L, "groups", None) is not None:
            c.groups = [(dofs, round_storage(inv, fmt).astype(np.float32)) for dofs, inv in L.groups]
        if L.weight is not None:
            c.weight = L.weight.astype(np.float32)
        if L.P is not None:
            c.P = L.P.astype(np.float32)
        h.levels.append(c)
    h.omega = np.float32(hierarchy.omega)
    lu = hierarchy.coarse_lu
    h.coarse_solve = lambda b: sla.lu_solve(lu, np.asarray(b, dtype=np.float64)).astype(np.float32)
    return h
