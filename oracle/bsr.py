"""Block-sparse matrices with n_c x n_c node blocks (Section 4.3), oracle side.

A level matrix is given as block rows over mesh nodes: ``row_ptr`` (nodes+1),
``col_idx`` (block columns) and ``vals`` (nnzb, n_c, n_c) with row-major
blocks.  The product y = A x is taken with scipy's BSR matrix, a library
primitive; ``block_lookup`` returns individual node blocks for the patch
extraction of the smoother.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class BlockMatrix:
    def __init__(self, row_ptr, col_idx, vals):
        self.row_ptr = np.asarray(row_ptr, dtype=np.int64)
        self.col_idx = np.asarray(col_idx, dtype=np.int64)
        self.vals = np.asarray(vals, dtype=np.float64)
        self.nodes = self.row_ptr.shape[0] - 1
        self.ncomp = self.vals.shape[1]
        n = self.nodes * self.ncomp
        self.csr = sp.bsr_matrix((self.vals, self.col_idx, self.row_ptr), shape=(n, n)).tocsr()
        rows = np.repeat(np.arange(self.nodes, dtype=np.int64), np.diff(self.row_ptr))
        keys = rows * self.nodes + self.col_idx
        order = np.argsort(keys, kind="stable")
        self._keys = keys[order]
        self._order = order

    @property
    def size(self) -> int:
        return self.nodes * self.ncomp

    def matvec(self, x: np.ndarray) -> np.ndarray:
        return self.csr @ x

    def dense(self) -> np.ndarray:
        return self.csr.toarray()

    def block_lookup(self, rows, cols) -> np.ndarray:
        """Blocks A_{rows, cols} (zero where the pattern has no block), shape (..., n_c, n_c)."""
        rows, cols = np.broadcast_arrays(np.asarray(rows, dtype=np.int64),
                                         np.asarray(cols, dtype=np.int64))
        q = (rows * self.nodes + cols).reshape(-1)
        pos = np.searchsorted(self._keys, q)
        pos_c = np.minimum(pos, self._keys.shape[0] - 1)
        hit = self._keys[pos_c] == q
        out = np.zeros((q.shape[0], self.ncomp, self.ncomp))
        out[hit] = self.vals[self._order[pos_c[hit]]]
        return out.reshape(rows.shape + (self.ncomp, self.ncomp))
