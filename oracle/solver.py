"""The whole oracle solve: FGMRES(m) preconditioned by one V(nu1, nu2) cycle.

Section 4.3: (I) GMRES outer iteration, (II) geometric multigrid V-cycle as
preconditioner, (III) Vanka smoother with omega_V = 0.8.  Stopping rule:
2-norm of the true residual relative to ||b||_2 (Section 5.5 states a
relative reduction; the norm is this build's reading).
"""

from __future__ import annotations

import time

import numpy as np

from .fgmres import fgmres
from .multigrid import Hierarchy


class OracleSolver:
    def __init__(self, levels, fine_mask, nu1=2, nu2=2, omega=0.8, weighting="average"):
        t0 = time.perf_counter()
        self.h = Hierarchy(levels, fine_mask, nu1=nu1, nu2=nu2, omega=omega, weighting=weighting)
        self.setup_seconds = time.perf_counter() - t0

    def solve(self, b, rtol=1e-8, restart=30, maxit=1000, history=None):
        A = self.h.fine.A
        return fgmres(A.matvec, self.h.vcycle, b, rtol=rtol, restart=restart, maxit=maxit,
                      history=history)


def solve(levels, fine_mask, b, rtol=1e-8, restart=30, maxit=1000, nu1=2, nu2=2, omega=0.8,
          weighting="average"):
    s = OracleSolver(levels, fine_mask, nu1=nu1, nu2=nu2, omega=omega, weighting=weighting)
    return s.solve(b, rtol=rtol, restart=restart, maxit=maxit)
