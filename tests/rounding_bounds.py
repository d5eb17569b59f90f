"""Per-entry rounding bounds for comparing the reduced-precision GPU path with
the FP64 oracle (test helper; imports nothing from the library).

One step of Eq. (vanka) in the FP32 / BF16 path, x1 = x0 + omega W sum_P
R_P^T A_P^{-1} R_P (b - A x0), computes the defect with the FP32 matrix, applies
the stored inverse (FP32 or BF16 entries) in FP32 arithmetic and accumulates
the patch corrections in FP32.  To first order in the unit roundoffs the
computed x1 differs from the exact step by at most, entry by entry,

    B = u |x0| + omega w sum_P R_P^T [ (u_s + (n_p + 2^d + 4) u) |A_P^-1| |d_P|
                                      + (k + 2) u |A_P^-1| (|b| + |A| |x0|)_P
                                      + e_inv max|A_P^-1| sum |d_P| ]

with u = 2^-24 (FP32 arithmetic, matrix and vector storage), u_s the unit
roundoff of the stored inverse (2^-24 for FP32, 2^-8 for BF16), n_p the patch
size, k = 3^d n_c the terms of one block row of A, and e_inv = 1e-7 the bound
on how far the library's FP64 Gauss-Jordan inverse may differ from the
oracle's LAPACK inverse relative to the largest entry (the FP64 patch-inverse
parity tolerance).  The terms are: one rounding of x0 + correction; the FP32
dot products of the apply (n_p terms) and the sum over at most 2^d patches
with the weight and omega; the FP32 defect (k products and b, plus the FP32
rounding of A); and the stored inverse itself.
"""

from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
U_STORE = {1: 2.0 ** -24, 2: 2.0 ** -8}      # by library precision code (FP32, BF16)
E_INV = 1e-7


def vanka_step_and_bound(inv, dofs, b, x0, d, abs_ax, weight, omega, prec, dim, nc):
    """Oracle step x1 (FP64) and its rounding bound B over the patches given by
    inv (P, n_p, n_p) and dofs (P, n_p); b, x0, d = b - A x0 and abs_ax =
    |A||x0| are full-length FP64 vectors.  Entries of x1 and B are exact only
    where every patch containing the unknown is among the given ones."""
    n_p = dofs.shape[1]
    k = 3 ** dim * nc
    u_s = U_STORE[prec]
    corr = np.zeros_like(x0)
    t1 = np.zeros_like(x0)
    t2 = np.zeros_like(x0)
    t3 = np.zeros_like(x0)
    dp = d[dofs]
    a_inv = np.abs(inv)
    np.add.at(corr, dofs, np.einsum("pij,pj->pi", inv, dp))
    np.add.at(t1, dofs, np.einsum("pij,pj->pi", a_inv, np.abs(dp)))
    np.add.at(t2, dofs, np.einsum("pij,pj->pi", a_inv, (np.abs(b) + abs_ax)[dofs]))
    per_patch = a_inv.reshape(a_inv.shape[0], -1).max(axis=1) * np.abs(dp).sum(axis=1)
    np.add.at(t3, dofs, np.repeat(per_patch[:, None], n_p, axis=1))
    x1 = x0 + omega * weight * corr
    bound = U32 * np.abs(x0) + omega * weight * (
        (u_s + (n_p + 2 ** dim + 4) * U32) * t1 + (k + 2) * U32 * t2 + E_INV * t3)
    return x1, bound


def vanka_groups_step_and_bound(groups, b, x0, d, abs_ax, weight, omega, prec, dim, nc):
    """vanka_step_and_bound for patches of several sizes: groups = [(dofs,
    inverses)] per size; the dot-product length term uses the largest patch."""
    n_p = max(dofs.shape[1] for dofs, _ in groups)
    k = 3 ** dim * nc
    u_s = U_STORE[prec]
    corr, t1, t2, t3 = (np.zeros_like(x0) for _ in range(4))
    for dofs, inv in groups:
        dp = d[dofs]
        a_inv = np.abs(inv)
        np.add.at(corr, dofs, np.einsum("pij,pj->pi", inv, dp))
        np.add.at(t1, dofs, np.einsum("pij,pj->pi", a_inv, np.abs(dp)))
        np.add.at(t2, dofs, np.einsum("pij,pj->pi", a_inv, (np.abs(b) + abs_ax)[dofs]))
        per_patch = a_inv.reshape(a_inv.shape[0], -1).max(axis=1) * np.abs(dp).sum(axis=1)
        np.add.at(t3, dofs, np.repeat(per_patch[:, None], dofs.shape[1], axis=1))
    x1 = x0 + omega * weight * corr
    bound = U32 * np.abs(x0) + omega * weight * (
        (u_s + (n_p + 2 ** dim + 4) * U32) * t1 + (k + 2) * U32 * t2 + E_INV * t3)
    return x1, bound


def to_storage32(a):
    """The FP32 value the test hands to the library, as FP64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def vcycle_tolerance(dz_model, z_max, nc):
    """Per-component tolerance of a reduced-precision V-cycle or multi-step
    smoothing against the FP64 oracle:

        tol_c = 8 max |dz_c| + 16 u max |z|

    dz is how far the oracle's cycle moves when run the reduced-precision way
    (oracle.precision.with_fp32_arithmetic: binary32 matrices, vectors and
    arithmetic, inverses rounded once to the storage format, exact coarse
    solve); its largest entry per component is dz_model (length nc).  Its
    summation orders differ from the library's, so it gives the size of the
    rounding errors, not their values; the factor 8 covers that.  The second
    term is a floor of a few binary32 roundings of the largest entry.  (The
    rounding errors of a component are not proportional to its own entries:
    the pressure, the largest entries, enters the velocity rows through the
    coupling blocks, and near-singular coarse corrections amplify the binary32
    residual's cancellation.)"""
    per = 8.0 * np.asarray(dz_model, dtype=np.float64) + 16.0 * U32 * float(z_max)
    return per.reshape(1, nc)


def model_vcycle_dz(h, r, fmt, nc):
    """Per-component largest |V_model(r) - V(r)| (see vcycle_tolerance) and V(r)."""
    from oracle.precision import with_fp32_arithmetic
    z = h.vcycle(r)
    zm = with_fp32_arithmetic(h, fmt).vcycle(np.asarray(r, dtype=np.float32)).astype(np.float64)
    return np.abs(zm - z).reshape(-1, nc).max(axis=0), z


def within(err, tol_comp, nc):
    """True where |err| (node-blocked vector) is within the per-component tolerance."""
    return np.abs(np.asarray(err).reshape(-1, nc)) <= tol_comp
