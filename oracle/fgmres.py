"""Right-preconditioned flexible GMRES(m), item (I) of Section 4.3 (oracle).

The paper runs GMRES without restarts (it converges in fewer than ten
steps); the reading here is flexible GMRES with restart length m, because the
preconditioner may be a reduced-precision V-cycle that is not the same linear
map at every step.  Modified Gram-Schmidt Arnoldi, Givens rotations on the
Hessenberg matrix; the iteration stops when the rotated residual estimate
|g_{j+1}| / ||b||_2 <= rtol, then forms x = x0 + Z y.  After each cycle the
true residual ||b - A x||_2 / ||b||_2 is recomputed; the solve ends when it is
<= rtol, otherwise it restarts from x.  The iteration count is the total
number of preconditioner applications.
"""

from __future__ import annotations

import math

import numpy as np


def givens(a: float, b: float):
    """(c, s) with [c s; -s c] [a; b] = [r; 0], r = hypot(a, b) >= 0."""
    if b == 0.0:
        return (1.0, 0.0) if a >= 0.0 else (-1.0, 0.0)
    r = math.hypot(a, b)
    return a / r, b / r


def fgmres(matvec, precond, b, rtol=1e-8, restart=30, maxit=1000, x0=None, history=None):
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    info = {"iterations": 0, "restarts": 0, "converged": False, "rel_residual": 0.0}
    if bnorm == 0.0:
        x[:] = 0.0
        info["converged"] = True
        return x, info
    its = 0
    cycle = 0
    while True:
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
        info["rel_residual"] = beta / bnorm
        if beta / bnorm <= rtol:
            info["converged"] = True
            break
        if its >= maxit:
            break
        if cycle > 0:
            info["restarts"] += 1
        cycle += 1
        m = restart
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = precond(V[j])
            Z.append(z)
            w = matvec(z)
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            for i in range(j):
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -sn[i] * hi + cs[i] * hi1
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            hjj, hj1 = H[j, j], H[j + 1, j]
            H[j, j] = cs[j] * hjj + sn[j] * hj1
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            est = abs(g[j + 1]) / bnorm
            if history is not None:
                history.append(est)
            breakdown = hj1 == 0.0
            if est <= rtol or its >= maxit or breakdown:
                break
            V.append(w / hj1)
        # back substitution H[:k,:k] y = g[:k]
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
    info["iterations"] = its
    return x, info
