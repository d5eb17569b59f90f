"""Convenience layer over the C ABI: owns one hierarchy handle.

It only marshals arguments (host numpy arrays for the level matrices and the
Dirichlet mask, tensors or arrays for vectors) and calls libnmg.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import nmg


def solve_opts(**kw) -> nmg.nmg_solve_opts:
    o = nmg.nmg_solve_opts()
    nmg.check(nmg.nmg_default_opts(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Session:
    """One multigrid hierarchy on the current CUDA device.

    levels: sequence (coarsest first) of (row_ptr int64, col_idx int32,
    vals float64 (nnzb, nc, nc)) host arrays; mask: uint8 finest-level
    Dirichlet mask; precisions: bit mask of nmg.NMG_PREC_* (0 = all); ncomp:
    unknowns per node, dim + 1 (default) or dim.
    """

    def __init__(self, dim, n, levels, mask, precisions=0, stream=None, mem_budget=0, nlevels=None, ncomp=None):
        self.dim = int(dim)
        self.n = tuple(int(v) for v in n)
        self._mask = np.ascontiguousarray(mask, dtype=np.uint8)
        d = nmg.nmg_mesh_desc()
        d.dim = self.dim
        for k in range(3):
            d.n[k] = self.n[k] if k < self.dim else 1
        d.levels = len(levels) if nlevels is None else int(nlevels)
        d.ncomp = self.dim + 1 if ncomp is None else int(ncomp)
        d.patch_cells = 2
        d.dirichlet_mask = self._mask.ctypes.data
        d.precisions = int(precisions)
        d.mem_budget_bytes = int(mem_budget)
        d.stream = stream
        self.handle = C.c_void_p()
        nmg.check(nmg.nmg_create_hierarchy(d, self.handle))
        for lev, (rp, ci, vals) in enumerate(levels):
            self.set_level(lev, rp, ci, vals)

    def set_level(self, lev, row_ptr, col_idx, vals):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        v = np.ascontiguousarray(vals, dtype=np.float64)
        nmg.check(nmg.nmg_set_jacobian(self.handle, lev, rp.shape[0] - 1, ci.shape[0], rp, ci, v, 0))

    def set_large_patches(self, cell_mask):
        """Large Vanka patches (4^d cells) over the flagged finest-level cells
        (numpy array in array order (z,) y, x, i.e. x fastest), or None."""
        m = None if cell_mask is None else np.ascontiguousarray(cell_mask, dtype=np.uint8)
        nmg.check(nmg.nmg_set_large_patches(self.handle, m))

    def patch_layout(self, level):
        ns, nl, ps, pl = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
        nmg.check(nmg.nmg_patch_layout(self.handle, level, ns, nl, ps, pl))
        return ns.value, nl.value, ps.value, pl.value

    def solve(self, b, x, **opts):
        info = nmg.nmg_solve_info()
        st = nmg.nmg_solve(self.handle, b, x, solve_opts(**opts), info)
        if st < 0 and st != nmg.NMG_ERR_NOT_CONVERGED:
            nmg.check(st)
        return info

    def solve_many(self, b, x, nrhs, **opts):
        """nrhs columns (column k at offset k * unknowns of b and x); returns the
        list of per-column nmg_solve_info records."""
        infos = (nmg.nmg_solve_info * nrhs)()
        st = nmg.nmg_solve_many(self.handle, nrhs, b, x, solve_opts(**opts), infos)
        if st < 0 and st != nmg.NMG_ERR_NOT_CONVERGED:
            nmg.check(st)
        return list(infos)

    def bytes(self) -> int:
        v = C.c_size_t()
        nmg.check(nmg.nmg_hierarchy_bytes(self.handle, v))
        return int(v.value)

    def close(self):
        if self.handle:
            nmg.nmg_destroy_hierarchy(self.handle)
            self.handle = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
